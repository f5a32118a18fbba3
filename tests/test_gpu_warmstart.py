"""The warm-start network on the GPU: forward and gradients against the FP64
numpy oracle (finite differences), and the trained network's gain over the
solve without it."""
import numpy as np
import pytest

import ep_inputs as E
import oracle as O
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


@pytest.mark.parametrize("nd,shape,base,levels,N", [(2, (36, 20), 16, 3, 2), (3, (12, 8, 20), 16, 2, 1),
                                                    (3, (16, 16, 16), 32, 3, 1)])
def test_tensor_core_forward_matches_the_bf16_input_oracle(P, nd, shape, base, levels, N):
    """The inference forward, whose 3^D convolutions with 16..128 output
    channels run as tcgen05 implicit GEMMs (BF16 inputs from TMA boxes, FP32
    accumulation in tensor memory), against the FP64 numpy network with the
    same BF16 rounding of those convolutions' inputs, on the warm start's
    channel counts (input channels padded to 16) and shapes whose bricks are
    ragged; the training forward (FP32 on CUDA cores) is checked through the
    loss against the unrounded network."""
    import torch
    cin, cout = P.warm_in(nd), P.warm_out(nd)
    net = P.Net(nd, cin, cout, base=base, levels=levels, seed=13)
    table, _ = U.layer_table(nd, cin, cout, base, levels)
    rng = np.random.default_rng(8)
    params = net.get_params().astype(np.float64)
    for (ci, co, k, wo, bo) in table:
        params[bo:bo + co] = rng.normal(size=co) * 0.05
    ci, co, k, wo, bo = table[-1]
    params[wo:wo + ci * co] = rng.normal(size=ci * co) * 0.3
    net.set_params(params.astype(np.float32))
    pk = params.copy()
    for (ci, co, k, wo, bo) in table:
        pk[wo:wo + ci * co * k ** nd] = _bf16(params[wo:wo + ci * co * k ** nd])
        pk[bo:bo + co] = params[bo:bo + co].astype(np.float32)
    dims = tuple(reversed(shape))
    x = rng.normal(size=(N, cin) + dims).astype(np.float32)
    t = rng.normal(size=(N, cout) + dims).astype(np.float32)
    xg = torch.tensor(x, device="cuda").contiguous()
    tg = torch.tensor(t, device="cuda").contiguous()
    yg = torch.full((N, cout) + dims, float("nan"), dtype=torch.float32, device="cuda")
    net.forward(xg.data_ptr(), N, list(shape), yg.data_ptr())
    torch.cuda.synchronize()
    y = yg.cpu().numpy().astype(np.float64)
    y_bf = U.forward(pk, x.astype(np.float64), nd, cin, cout, base, levels, bf16_inputs=True)
    y_fp = U.forward(pk, x.astype(np.float64), nd, cin, cout, base, levels)
    scale = np.abs(y_bf).max()
    err_bf = np.abs(y - y_bf).max() / scale
    err_fp = np.abs(y - y_fp).max() / scale
    assert np.isfinite(y).all() and scale > 0
    # FP32 accumulation in another order can move an intermediate value
    # across a BF16 rounding boundary (one unit of 2^-8 relative), which the
    # following layers carry on: a few 1e-3 of the output scale
    assert err_bf <= 6e-3, (err_bf, err_fp)
    assert err_bf < err_fp          # the BF16 input model explains most of the difference
    loss = net.loss(xg.data_ptr(), tg.data_ptr(), N, list(shape))
    ref = U.loss(pk, x.astype(np.float64), t.astype(np.float64), nd, cin, cout, base, levels)
    assert abs(loss - ref) <= 1e-4 * ref
    net.close()


def _lockstep(P, s, incs, coarsens):
    """A GPU FP64 grid and the oracle through `incs` increments; then the
    GPU's features before the next increment and its targets after it,
    against the numpy definition fed with the GPU's fields and the oracle's
    physical response of the converged velocity (with the old history)."""
    import torch
    from oracle import warm_oracle as WO
    nd = s.ndim
    rates = [s.a, -s.a] if nd == 2 else [s.a, 0.0, -s.a]
    g = P.Grid(nd, s.n, s.L, precision=P.FP64)
    g.set_material(s.K, s.G, s.mu_s, s.phi_deg, s.psi_deg, s.cohesion())
    g.set_solver(tol=s.tol)
    g.warm_record(True)
    o = O.from_setup(s, tol=s.tol)
    vn = ["vx", "vy", "vz"][:nd]
    tn_names = ["txx", "tyy", "tzz"][:nd]
    ts_names = ["txy"] if nd == 2 else ["txy", "txz", "tyz"]
    vs = []
    for _ in range(incs):
        g.apply_increment_rates(rates, s.dt)
        g.solve_increment()
        o.apply_increment(rates, s.dt)
        o.solve_increment()
        vs.append([g.get(v) for v in vn])
    assert (g.get("scale") < 1).any()
    old = {k: g.get(k) for k in tn_names + ts_names + ["p", "scale", "coh", "epl"]}
    feats = {}
    for f in coarsens:
        nv = int(np.prod(g.warm_dims(f)))
        x = torch.zeros(P.warm_in(nd) * nv, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()   # the library writes on its own (non-blocking) stream
        g.warm_features(x.data_ptr(), f)
        torch.cuda.synchronize()
        f_np = WO.features(s.n, f, vs[-1], vs[-2], [old[k] for k in tn_names], [old[k] for k in ts_names],
                           old["p"], old["scale"], old["coh"], old["epl"], rates, s.L[:nd], s.dt, s.G)
        np.testing.assert_allclose(x.cpu().numpy(), f_np, rtol=1e-5, atol=1e-6)
        feats[f] = f_np
    g.apply_increment_rates(rates, s.dt)
    info = g.solve_increment()
    assert info["n_plastic"] > 0
    v_new = [g.get(v) for v in vn]
    o.apply_increment(rates, s.dt)
    o.eval(np.concatenate([a.ravel() for a in v_new]))
    phys = {k: o.eval_stress(k) for k in tn_names + ts_names}
    for f in coarsens:
        nv = int(np.prod(g.warm_dims(f)))
        t = torch.zeros(P.warm_out(nd) * nv, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        g.warm_target(t.data_ptr(), f)
        torch.cuda.synchronize()
        t_np = WO.target(s.n, f, v_new, vs[-1], [g.get(k) for k in tn_names], [g.get(k) for k in ts_names],
                         [phys[k] for k in tn_names], [phys[k] for k in ts_names], rates, s.L[:nd], s.dt, s.G)
        tg = t.cpu().numpy()
        np.testing.assert_allclose(tg, t_np, rtol=1e-4, atol=2e-5 * max(1.0, np.abs(t_np).max()))
        assert np.abs(t_np).max() > 0
    g.close()


def test_features_and_targets_match_their_numpy_definition_2d(P):
    """The feature and target kernels against their plain numpy definition
    (oracle/warm_oracle.py) on a 2D FP64 grid past first yield, on the fine
    grid and coarsened by 2 and 4 (ragged coarse cells)."""
    s = E.config(1, n=(30, 26), L=(1.0, 26 / 30), tol=1e-9)
    _lockstep(P, s, 7, (1, 2, 4))


def test_features_and_targets_match_their_numpy_definition_3d(P):
    """The same on a 3D FP64 box (x-z pure shear) coarsened by 1, 2 and 3."""
    s = E.config(3, n=(12, 10, 9), inclusion_radius=0.25, tol=1e-9)
    _lockstep(P, s, 6, (1, 2, 3))


def test_output_scale_scales_the_output_and_its_gradient(P):
    """With an output scale s the network's output is s times its head's, the
    loss is taken in units of s, and the gradient is that loss's (finite
    differences of the numpy network with its output times s)."""
    import torch
    nd, shape, base, levels, N = 2, (8, 8), 2, 2, 2
    cin, cout = nd + 2, nd
    net = P.Net(nd, cin, cout, base=base, levels=levels, seed=3)
    table, _ = U.layer_table(nd, cin, cout, base, levels)
    rng = np.random.default_rng(2)
    params = net.get_params().astype(np.float64)
    ci, co, k, wo, bo = table[-1]
    params[wo:wo + ci * co] = rng.normal(size=ci * co) * 0.3
    net.set_params(params.astype(np.float32))
    pk = params.copy()
    for (ci, co, k, wo, bo) in table:
        pk[wo:wo + ci * co * k ** nd] = _bf16(params[wo:wo + ci * co * k ** nd])
        pk[bo:bo + co] = params[bo:bo + co].astype(np.float32)
    dims = tuple(reversed(shape))
    x = rng.normal(size=(N, cin) + dims).astype(np.float32)
    t = rng.normal(size=(N, cout) + dims).astype(np.float32)
    xg = torch.tensor(x, device="cuda").contiguous()
    tg = torch.tensor(t, device="cuda").contiguous()
    y1 = torch.empty((N, cout) + dims, dtype=torch.float32, device="cuda")
    y2 = torch.empty_like(y1)
    net.forward(xg.data_ptr(), N, list(shape), y1.data_ptr())
    net.set_output_scale(0.37)
    net.forward(xg.data_ptr(), N, list(shape), y2.data_ptr())
    torch.cuda.synchronize()
    np.testing.assert_allclose(y2.cpu().numpy(), 0.37 * y1.cpu().numpy(), rtol=1e-6, atol=1e-7)
    loss, g = net.gradients(xg.data_ptr(), tg.data_ptr(), N, list(shape))
    xr, tr = x.astype(np.float64), t.astype(np.float64)

    def scaled_loss(p):      # the loss in units of the scale
        return float(np.mean(((0.37 * U.forward(p, xr, nd, cin, cout, base, levels) - tr) / 0.37) ** 2))

    assert abs(loss - scaled_loss(pk)) <= 1e-4 * loss
    g_ref = np.zeros_like(pk)
    for i in range(pk.size):
        a, b = pk.copy(), pk.copy()
        a[i] += 1e-5
        b[i] -= 1e-5
        g_ref[i] = (scaled_loss(a) - scaled_loss(b)) / 2e-5
    assert np.abs(g - g_ref).max() <= 5e-3 * np.abs(g_ref).max()
    net.close()


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
        out.append(E.Setup("ws%d" % sd, 2, n, phi_deg=25.0 + 2 * (q % 4), c0=1.3e-3 + 1e-4 * (q % 4),
                           inclusion_radius=0.08, inclusion_centre=(0.03 * ((q % 5) - 2), -0.02 * ((q % 3) - 1), 0.0),
                           seed=sd, tol=1e-6))
    return out


def _grid(P, s):
    g = P.Grid(2, s.n, precision=P.FP32_MIXED)
    g.set_material(s.K, s.G, s.mu_s, s.phi_deg, s.psi_deg, s.cohesion())
    g.set_solver(tol=s.tol, max_iter=2000000)
    return g


def test_trained_warm_start_cuts_iterations(P):
    """Train on the trajectories of six setups, then follow three held-out
    setups.  From the third increment on, each increment is solved from the
    same committed state (device checkpoint) three times: started by the
    trained network, by a zero network and from the plain start.  The zero
    network reproduces the plain start exactly (same iterations); all reach
    the tolerance, and the trained network's starts need fewer iterations in
    total than the zero network's.  Before the band forms (increments 3-5)
    the answers agree closely; afterwards the increment's problem is nearly
    singular in the band and two starts may stop at answers that differ well
    above the tolerance (the non-uniqueness of a localizing solution), so
    there the difference is only reported."""
    from paper_2305_01701_gb300 import warmstart as W
    incs = 12
    train_setups = _setups(range(101, 107))
    test_setups = _setups([201, 202, 203])
    net = W.new_net(2, base=16, levels=3, seed=7)
    zero = W.new_net(2, base=16, levels=3, seed=7)
    data = W.Samples(2, (48, 48, 1), capacity=len(train_setups) * incs)
    for s in train_setups:
        g = _grid(P, s)
        W.collect(g, 1.0, s.dt, incs, data)
        g.close()
    assert data.n == len(train_setups) * (incs - 2)
    losses = W.train(net, [data], steps=800, lr=1e-3, batch=8)
    assert np.mean(losses[-50:]) < 0.5 * np.mean(losses[:50])
    tot = {"trained": 0, "zero": 0, "plain": 0}
    worst, early = 0.0, 0.0
    for s in test_setups:
        g = _grid(P, s)
        for inc in range(1, incs + 1):
            if inc >= 3:
                g.snapshot()
                out, txx = {}, {}
                for name, nn in (("trained", net), ("zero", zero)):
                    g.attach_warm_start(nn)
                    g.apply_increment(1.0, s.dt, P.LOAD_XY, use_warm_start=True)
                    out[name] = g.solve_increment()
                    txx[name] = g.get("txx")
                    g.restore()
                g.apply_increment(1.0, s.dt, P.LOAD_XY)
                out["plain"] = g.solve_increment()
                txx["plain"] = g.get("txx")
                assert out["zero"]["iters"] == out["plain"]["iters"]
                assert np.array_equal(txx["zero"], txx["plain"])
                for k in tot:
                    assert out[k]["eps_res"] <= s.tol
                    tot[k] += out[k]["iters"]
                d = np.abs(txx["trained"] - txx["plain"]).max() / np.abs(txx["plain"]).max()
                if inc <= 5:
                    early = max(early, d)
                worst = max(worst, d)
            else:
                g.apply_increment(1.0, s.dt, P.LOAD_XY)
                g.solve_increment()
        g.close()
    print("iterations", tot, "txx difference before the band", early, "worst", worst)
    assert tot["trained"] < tot["zero"]
    assert early < 1e-4
