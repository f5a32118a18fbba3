"""The warm-start network on the GPU: forward and gradients against the FP64
numpy oracle (finite differences), and the trained network's gain over the
solve without it."""
import numpy as np
import pytest

import ep_inputs as E
from oracle import unet_oracle as U

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


def _bf16(a):
    """Round FP32 values to BF16 (nearest even), as the kernels read weights."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    r = ((b >> 16) & 1) + 0x7FFF
    return ((b + r) & 0xFFFF0000).astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("nd,shape,base,levels", [(2, (8, 12), 3, 2), (2, (8, 8), 2, 3), (3, (4, 4, 8), 2, 2)])
def test_net_forward_and_gradient_match_oracle(P, nd, shape, base, levels):
    import torch
    cin, cout, N = nd + 2, nd, 2
    net = P.Net(nd, cin, cout, base=base, levels=levels, seed=11)
    params = net.get_params().astype(np.float64)
    table, n = U.layer_table(nd, cin, cout, base, levels)
    assert n == params.size
    # give the zero-initialised head weights values so every path carries gradient
    rng = np.random.default_rng(5)
    ci, co, k, wo, bo = table[-1]
    params[wo:wo + ci * co] = rng.normal(size=ci * co) * 0.3
    params[bo:bo + co] = rng.normal(size=co) * 0.1
    net.set_params(params.astype(np.float32))
    # the kernels use BF16 weights and FP32 biases
    pk = params.copy()
    for (ci, co, k, wo, bo) in table:
        pk[wo:wo + ci * co * k ** nd] = _bf16(params[wo:wo + ci * co * k ** nd])
        pk[bo:bo + co] = params[bo:bo + co].astype(np.float32)
    xs = (N, cin) + tuple(reversed(shape))
    x = rng.normal(size=xs)
    t = rng.normal(size=(N, cout) + tuple(reversed(shape)))
    xg = torch.tensor(x, dtype=torch.float32, device="cuda").contiguous()
    tg = torch.tensor(t, dtype=torch.float32, device="cuda").contiguous()
    yg = torch.empty((N, cout) + tuple(reversed(shape)), dtype=torch.float32, device="cuda")
    net.forward(xg.data_ptr(), N, list(shape), yg.data_ptr())
    torch.cuda.synchronize()
    y_ref = U.forward(pk, x.astype(np.float32).astype(np.float64), nd, cin, cout, base, levels)
    np.testing.assert_allclose(yg.cpu().numpy(), y_ref, rtol=2e-4, atol=2e-4 * np.abs(y_ref).max())
    loss, g = net.gradients(xg.data_ptr(), tg.data_ptr(), N, list(shape))
    xr = x.astype(np.float32).astype(np.float64)
    tr = t.astype(np.float32).astype(np.float64)
    assert abs(loss - U.loss(pk, xr, tr, nd, cin, cout, base, levels)) <= 1e-4 * loss
    assert net.loss(xg.data_ptr(), tg.data_ptr(), N, list(shape)) == loss   # the same pass, no gradient copy
    g_ref = U.fd_gradient(pk, xr, tr, nd, cin, cout, base, levels, h=1e-5)
    scale = np.abs(g_ref).max()
    assert np.abs(g - g_ref).max() <= 5e-3 * scale, (np.abs(g - g_ref).max(), scale)
    net.close()


def test_features_and_targets_match_their_numpy_definition(P):
    """The feature and target kernels against their plain numpy definition
    (oracle/warm_oracle.py) on a 2D FP64 grid past first yield (so the scale
    channel varies): the scale S exactly, every channel within FP32
    rounding."""
    import torch
    from oracle import warm_oracle as WO
    s = E.config(1, n=(30, 26), tol=1e-9)
    g = P.Grid(2, s.n, precision=P.FP64)
    g.set_material(s.K, s.G, s.mu_s, s.phi_deg, s.psi_deg, s.cohesion())
    g.set_solver(tol=s.tol)
    vs = []
    for _ in range(7):
        g.apply_increment(1.0, s.dt, P.LOAD_XY)
        g.solve_increment()
        vs.append([g.get("vx"), g.get("vy")])
    assert (g.get("scale") < 1).any()
    nv = int(np.prod(g.warm_dims()))
    x = torch.zeros(4 * nv, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()   # the library writes on its own (non-blocking) stream
    S = g.warm_features(x.data_ptr())
    torch.cuda.synchronize()
    f_np, S_np = WO.features(s.n, vs[-1], vs[-2], g.get("scale"), s.cohesion())
    assert S == S_np
    f_gpu = x.cpu().numpy()
    np.testing.assert_allclose(f_gpu, f_np, rtol=1e-6, atol=1e-7)
    g.apply_increment(1.0, s.dt, P.LOAD_XY)
    g.solve_increment()
    t = torch.zeros(2 * nv, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    g.warm_target(x.data_ptr(), S, t.data_ptr())
    t_np = WO.target(s.n, [g.get("vx"), g.get("vy")], vs[-1], S, f_gpu)
    np.testing.assert_allclose(t.cpu().numpy(), t_np, rtol=1e-5, atol=1e-6)
    g.close()


def test_training_reduces_the_loss(P):
    import torch
    rng = np.random.default_rng(0)
    net = P.Net(2, 4, 2, base=8, levels=3, seed=3)
    x = torch.tensor(rng.normal(size=(4, 4, 16, 16)), dtype=torch.float32, device="cuda").contiguous()
    # a learnable target: a smoothed copy of the first two channels
    t = (0.5 * x[:, :2]).contiguous()
    losses = [net.train_step(x.data_ptr(), t.data_ptr(), 4, [16, 16], 3e-3) for _ in range(200)]
    assert losses[-1] < 0.3 * losses[0], (losses[0], losses[-1])


def _setups(seeds, n=(48, 48)):
    out = []
    for q, sd in enumerate(seeds):
        out.append(E.Setup("ws%d" % sd, 2, n, phi_deg=25.0 + 2 * q, c0=1.3e-3 + 1e-4 * q, inclusion_radius=0.08,
                           inclusion_centre=(0.03 * q, -0.02 * q, 0.0), seed=sd, tol=1e-6))
    return out


def _grid(P, s):
    g = P.Grid(2, s.n, precision=P.FP32_MIXED)
    g.set_material(s.K, s.G, s.mu_s, s.phi_deg, s.psi_deg, s.cohesion())
    g.set_solver(tol=s.tol, max_iter=2000000)
    return g


def test_trained_warm_start_cuts_iterations(P):
    """Train on trajectories of four setups, then follow two held-out setups.
    From the third increment on, each increment is solved twice from the same
    committed state (device checkpoint): once started by the network, once
    from the plain start.  Both reach the tolerance and the warm starts need
    fewer iterations in total.  Before the band forms (increments 3-5, which
    converge in a few hundred iterations) the two answers agree closely;
    afterwards the increment's problem is nearly singular in the band and
    two starts may stop at answers that differ well above the tolerance (the
    non-uniqueness of a localizing solution), so there the difference is
    only reported."""
    from paper_2305_01701_gb300 import warmstart as W
    incs = 14
    train_setups = _setups([101, 102, 103, 104])
    test_setups = _setups([201, 202])
    net = W.new_net(2, base=16, levels=3, seed=7)
    dims = ((48 + 3) // 4 * 4, (48 + 3) // 4 * 4, 1)
    data = W.Samples(2, dims, capacity=len(train_setups) * incs)
    for s in train_setups:
        g = _grid(P, s)
        W.collect(g, 1.0, s.dt, incs, data)
        g.close()
    assert data.n == len(train_setups) * (incs - 2)
    losses = W.train(net, [data], steps=600, lr=1e-3, batch=8)
    assert np.mean(losses[-50:]) < np.mean(losses[:50])
    plain, warm, worst, early = 0, 0, 0.0, 0.0
    for s in test_setups:
        g = _grid(P, s)
        g.attach_warm_start(net)
        for inc in range(1, incs + 1):
            both = inc >= 3
            if both:
                g.snapshot()
                g.apply_increment(1.0, s.dt, P.LOAD_XY, use_warm_start=True)
                iw = g.solve_increment()
                tw = g.get("txx")
                g.restore()
            g.apply_increment(1.0, s.dt, P.LOAD_XY)
            ip = g.solve_increment()
            if both:
                assert max(iw["eps_res"], ip["eps_res"]) <= s.tol
                warm += iw["iters"]
                plain += ip["iters"]
                tp = g.get("txx")
                d = np.abs(tw - tp).max() / np.abs(tp).max()
                if inc <= 5:
                    early = max(early, d)
                worst = max(worst, d)
        g.close()
    print("plain", plain, "warm", warm, "txx difference before the band", early, "worst", worst)
    assert warm < plain
    assert early < 1e-4
