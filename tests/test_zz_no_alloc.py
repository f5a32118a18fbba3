"""The allocation-free forward of the warm-start network against the
allocating one, through the C ABI: same output, bit for bit, on calls in a
row (the shared static activation array carries nothing from one call to the
next), no change of the device's free memory across calls (it allocates
nothing), and a clear error above the static limit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_01701_gb300 import build as B
    B.build()
    import paper_2305_01701_gb300 as P
    return P


def _net(P, nd, base, levels, seed):
    cin, cout = nd + 2, nd
    net = P.Net(nd, cin, cout, base=base, levels=levels, seed=seed)
    params = net.get_params()
    rng = np.random.default_rng(seed)
    # give the zero-initialised head values so the output is not trivially zero
    params[-(base * cout + cout):] = rng.normal(size=base * cout + cout).astype(np.float32) * 0.3
    net.set_params(params)
    return net


@pytest.mark.parametrize("nd,shape,N,base,levels", [(2, (48, 40), 2, 16, 3), (3, (16, 8, 12), 1, 8, 3)])
def test_static_forward_matches_allocating_forward(P, nd, shape, N, base, levels):
    import torch
    net = _net(P, nd, base, levels, seed=21)
    cin, cout = nd + 2, nd
    dims = tuple(reversed(shape))
    rng = np.random.default_rng(4)
    for call in range(2):
        x = torch.tensor(rng.normal(size=(N, cin) + dims), dtype=torch.float32, device="cuda").contiguous()
        y_ref = torch.empty((N, cout) + dims, dtype=torch.float32, device="cuda")
        y_st = torch.full((N, cout) + dims, float("nan"), dtype=torch.float32, device="cuda")
        net.forward(x.data_ptr(), N, list(shape), y_ref.data_ptr())
        net.forward_static(x.data_ptr(), N, list(shape), y_st.data_ptr())
        torch.cuda.synchronize()
        assert torch.isfinite(y_ref).all()
        assert torch.equal(y_ref, y_st), (call, (y_ref - y_st).abs().max().item())
    net.close()


def test_static_forward_rejects_shapes_above_the_limit(P):
    import torch
    net = _net(P, 2, 32, 3, seed=3)
    x = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(P.EPError, match="static limit"):
        net.forward_static(x.data_ptr(), 1, [1024, 1024], x.data_ptr())
    net.close()


def test_static_forward_allocates_no_device_memory(P):
    """After one call has made the library's static array resident, further
    calls -- on a new network and at a new shape -- leave the device's free
    memory unchanged: the entry point allocates nothing."""
    import torch
    rng = np.random.default_rng(9)
    net0 = _net(P, 2, 16, 3, seed=5)
    x0 = torch.tensor(rng.normal(size=(1, 4, 32, 32)), dtype=torch.float32, device="cuda").contiguous()
    y0 = torch.empty((1, 2, 32, 32), dtype=torch.float32, device="cuda")
    net0.forward_static(x0.data_ptr(), 1, [32, 32], y0.data_ptr())
    torch.cuda.synchronize()
    net = _net(P, 2, 16, 3, seed=6)
    x = torch.tensor(rng.normal(size=(2, 4, 40, 48)), dtype=torch.float32, device="cuda").contiguous()
    y = torch.empty((2, 2, 40, 48), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        net.forward_static(x.data_ptr(), 2, [48, 40], y.data_ptr())
        net0.forward_static(x0.data_ptr(), 1, [32, 32], y0.data_ptr())
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.isfinite(y).all()
    net.close()
    net0.close()
