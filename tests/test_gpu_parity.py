"""GPU path (through the C ABI) against the FP64 CPU oracle.

FP64: every field within 1e-10 of the oracle, L-infinity normalised
(max|gpu - oracle| / max|oracle|, since pointwise ratios are undefined at
zeros), and the same iteration counts.  FP32 mixed: the stated bounds of
1e-5 on stress and 1e-4 on plastic strain (L-infinity normalised).
Sizes span several thread blocks and ragged edges (odd, non-square grids).
"""
import math

import numpy as np
import pytest

import ep_inputs as E
import oracle as O

pytestmark = pytest.mark.gpu

FIELDS_2D = ("vx", "vy", "txx", "tyy", "txy", "p", "epl", "ux", "uy", "exx", "eyy", "exy")
FIELDS_3D = ("vx", "vy", "vz", "txx", "tyy", "tzz", "txy", "txz", "tyz", "p", "epl", "ux", "uy", "uz",
             "exx", "eyy", "ezz", "exy", "exz", "eyz")


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_01701_gb300 import build as B
    B.build()
    import paper_2305_01701_gb300 as P
    return P


def rel_err(a, b, scale=0.0):
    """max|a - b| / max(max|b|, scale)."""
    den = max(np.abs(b).max(), scale)
    return np.abs(a - b).max() / den if den > 0 else np.abs(a - b).max()


GROUPS = {"stress": ("txx", "tyy", "tzz", "txy", "txz", "tyz", "p"), "velocity": ("vx", "vy", "vz"),
          "displacement": ("ux", "uy", "uz"), "strain": ("exx", "eyy", "ezz", "exy", "exz", "eyz"),
          "plastic": ("epl",)}


def group_scales(o, fields):
    """L-infinity scale of each field's physical group, from the oracle: a
    field is normalised by the largest component of its group (a pressure
    that is zero up to rounding is judged against the stress magnitude)."""
    sc = {}
    for names in GROUPS.values():
        present = [f for f in names if f in fields]
        m = max([np.abs(o.get(f)).max() for f in present] + [0.0])
        for f in present:
            sc[f] = m
    return sc


def rates_of(s):
    return [s.a, -s.a] if s.ndim == 2 else ([s.a, -s.a, 0.0] if s.load_plane == "xy" else [s.a, 0.0, -s.a])


def gpu_grid(P, s, precision, **solver):
    g = P.Grid(s.ndim, s.n, s.L, precision=precision)
    g.set_material(s.K, s.G, s.mu_s, s.phi_deg, s.psi_deg, s.cohesion())
    kw = dict(tol=s.tol)
    kw.update(solver)
    g.set_solver(**kw)
    return g


def run_pair(P, s, increments, precision=None, fields=None, tol_fields=1e-10, same_iters=True, **solver):
    precision = P.FP64 if precision is None else precision
    g = gpu_grid(P, s, precision, **solver)
    o = O.from_setup(s, **solver)
    fields = fields or (FIELDS_2D if s.ndim == 2 else FIELDS_3D)
    worst = {}
    for inc in range(1, increments + 1):
        g.apply_increment_rates(rates_of(s), s.dt)
        ig = g.solve_increment()
        o.apply_increment(rates_of(s), s.dt)
        io = o.solve_increment()
        if same_iters:
            assert ig["iters"] == io["iters"], (inc, ig, io)
        if tol_fields is not None:   # the line integrals of sigma_xx (G15)
            iscale = max(np.abs(o.get("txx")).max(), np.abs(o.get("p")).max()) * max(s.L)
            for k in ("sxx_int_centre", "sxx_int_right"):
                assert abs(ig[k] - io[k]) <= tol_fields * max(abs(io[k]), iscale), (inc, k, ig[k], io[k])
        assert ig["n_plastic"] == io["n_plastic"] or not same_iters, (inc, ig["n_plastic"], io["n_plastic"])
        sc = group_scales(o, fields)
        for f in fields:
            e = rel_err(g.get(f), o.get(f), sc[f])
            worst[f] = max(worst.get(f, 0.0), e)
            if tol_fields is not None:
                assert e <= tol_fields, (inc, f, e)
    g.close()
    return worst


def test_homogeneous_elastic_closed_form_2d(P):
    s = E.config(1, n=(37, 29), noise=0.0, inclusion_radius=0.0, c0=1.0)
    g = gpu_grid(P, s, P.FP64)
    for inc in range(1, 4):
        g.apply_increment(1.0, 1e-4, P.LOAD_XY)
        info = g.solve_increment()
        assert info["iters"] == 0
        np.testing.assert_allclose(g.get("txx"), 2e-4 * inc, rtol=1e-13)
        np.testing.assert_allclose(g.get("tyy"), -2e-4 * inc, rtol=1e-13)
        assert np.abs(g.get("txy")).max() < 1e-18


def test_fp64_parity_2d_inclusion_through_first_yield(P):
    """2D weak inclusion with noise, 40x33 cells (ragged), through the first
    plastic increments: iteration counts equal, every field <= 1e-10."""
    s = E.config(1, n=(40, 33))
    run_pair(P, s, 8)


def test_fp64_parity_2d_64_config1_first_increments(P):
    s = E.config(1)
    run_pair(P, s, 7)


def test_fp64_parity_2d_maxwell(P):
    """Visco-elasto-plastic (mu_s / (G dt) = 10) on a ragged 48x35 grid."""
    s = E.config(2, n=(48, 35), increments=14)
    run_pair(P, s, 14)


def test_fp64_parity_fixed_iterations_2d(P):
    """A deliberately unconverged fixed-iteration solve (tol 0, 300 iterations)
    on the first plastic increment compares the raw iteration with the
    oracle's, state included."""
    s = E.config(1, n=(33, 31), tol=1e-10)
    g = gpu_grid(P, s, P.FP64)
    o = O.from_setup(s)
    for inc in range(1, 6):
        if inc == 5:
            g.set_solver(tol=0.0, max_iter=300, n_chk=100)
            o.set_solver(tol=0.0, max_iter=300, n_chk=100)
        g.apply_increment(1.0, s.dt, P.LOAD_XY)
        o.apply_increment([1.0, -1.0], s.dt)
        ig = g.solve_increment(raise_on_fail=False)
        io = o.solve_increment(commit=False, raise_on_fail=False)
        if ig["status"] != 0:
            g.commit_increment()
        if io["status"] != 0:
            o.commit()
        else:
            o.commit()
        assert ig["iters"] == io["iters"], inc
    assert ig["status"] == 5 and io["status"] == 5
    sc = group_scales(o, FIELDS_2D)
    for f in FIELDS_2D:
        assert rel_err(g.get(f), o.get(f), sc[f]) <= 1e-11, f


def test_fp64_parity_3d_ragged(P):
    """3D x-z pure shear with a spherical inclusion on a ragged 17x13x11 grid."""
    s = E.config(3, n=(17, 13, 11), tol=1e-9, precision="fp64", inclusion_radius=0.15)
    run_pair(P, s, 8)


def test_fp64_parity_3d_xy_loading_jaumann_off(P):
    s = E.config(3, n=(12, 14, 10), tol=1e-9, precision="fp64", load_plane="xy", inclusion_radius=0.2)
    run_pair(P, s, 7, jaumann=False)


def test_fp64_parity_tiny_and_degenerate_grids(P):
    """1x1 (no interior faces), 2x2, 3x1 and 1x1x1 / 2x2x2."""
    for nd, n in ((2, (1, 1)), (2, (2, 2)), (2, (3, 1)), (3, (1, 1, 1)), (3, (2, 2, 2))):
        s = E.Setup("tiny", nd, n, inclusion_radius=0.0, noise=0.01, seed=5, tol=1e-11,
                    load_plane="xz" if nd == 3 else "xy")
        run_pair(P, s, 9)


def test_fp64_body_force_manufactured(P):
    sp = pytest.importorskip("sympy")
    from test_oracle_pins import _mms_2d
    (vxe, vye), (bx, by), dt = _mms_2d(24)
    s = E.Setup("mms", 2, (24, 24), c0=1.0, inclusion_radius=0.0, noise=0.0, tol=1e-11, dt=dt)
    g = gpu_grid(P, s, P.FP64)
    o = O.from_setup(s)
    g.apply_increment_rates([1.0, -1.0], dt, body_force=(bx, by))
    o.apply_increment([1.0, -1.0], dt, body_force=(bx, by))
    ig, io = g.solve_increment(), o.solve_increment()
    assert ig["iters"] == io["iters"]
    fl = ("vx", "vy", "txx", "tyy", "txy", "p")
    sc = group_scales(o, fl)
    for f in fl:
        assert rel_err(g.get(f), o.get(f), sc[f]) <= 1e-10, f
    del sp


def run_fp32_vs_oracle(P, s, increments, gpu_tol=1e-6, oracle_tol=1e-10, kernel=None, **solver):
    """FP32 mixed GPU solve at its tolerance against a tightly converged FP64
    oracle: the worst L-infinity-normalised error of each field."""
    g = gpu_grid(P, s, P.FP32_MIXED, tol=gpu_tol, max_iter=400000, **solver)
    if kernel is not None:
        g.set_kernel(*kernel)
    o = O.from_setup(s, tol=oracle_tol, **solver)
    fields = FIELDS_2D if s.ndim == 2 else FIELDS_3D
    worst = {}
    for inc in range(1, increments + 1):
        g.apply_increment_rates(rates_of(s), s.dt)
        g.solve_increment()
        o.apply_increment(rates_of(s), s.dt)
        o.solve_increment()
        sc = group_scales(o, fields)
        for f in fields:
            worst[f] = max(worst.get(f, 0.0), rel_err(g.get(f), o.get(f), sc[f]))
    worst["epl_max"] = float(np.abs(o.get("epl")).max())
    g.close()
    return worst


def test_fp32_mixed_within_stated_bounds_2d(P):
    """FP32 sweeps with FP64 norms and history: stress within 1e-5 and plastic
    strain within 1e-4 of the FP64 oracle (L-infinity normalised)."""
    s = E.config(1, n=(48, 40))
    worst = run_fp32_vs_oracle(P, s, 8)
    for f in ("txx", "tyy", "txy", "p"):
        assert worst[f] <= 1e-5, (f, worst[f])
    assert worst["epl"] <= 1e-4, worst["epl"]


@pytest.mark.parametrize("tile", [0, 3, 4])
def test_fp32_fused2d_within_stated_bounds(P, tile):
    """The fused 2D kernels in FP32 (block tile, warp strips of 64 and 32
    rows; the strips take untested clamped loads and the reciprocal-square-
    root return) against the FP64 oracle within the stated bounds."""
    s = E.config(1, n=(60, 90), inclusion_radius=0.08)
    worst = run_fp32_vs_oracle(P, s, 6, kernel=(P.KERNEL_FUSED, tile))
    for f in ("txx", "tyy", "txy", "p"):
        assert worst[f] <= 1e-5, (f, worst[f])
    assert worst["epl"] <= 1e-4, worst["epl"]


def test_fp32_mixed_within_stated_bounds_3d(P):
    s = E.config(3, n=(16, 15, 14), inclusion_radius=0.15)
    worst = run_fp32_vs_oracle(P, s, 7)
    for f in ("txx", "tyy", "tzz", "txy", "txz", "tyz", "p"):
        assert worst[f] <= 1e-5, (f, worst[f])
    assert worst["epl"] <= 1e-4, worst["epl"]


def test_fp32_register_kernel_interior_windows_against_oracle(P):
    """The benchmarked FP32 3D sweep (register z-march) on a grid with several
    interior windows, whose copy of the body skips the domain-boundary tests
    and takes untested clamped loads, against the FP64 oracle through first
    yield of the inclusion (which lies inside those windows): stress within
    1e-5 and plastic strain within 1e-4.  A window is 32 x 16 columns with
    28 x 12 written; on 90 x 40 columns the windows at x-blocks 1-2 and
    y-blocks 1-2 are interior."""
    nx, ny, nz = 90, 40, 24
    s = E.config(3, n=(nx, ny, nz), L=(1.0, ny / nx, nz / nx), inclusion_radius=0.06)
    worst = run_fp32_vs_oracle(P, s, 6, kernel=(P.KERNEL_FUSED_REG, 0))
    for f in ("txx", "tyy", "tzz", "txy", "txz", "tyz", "p"):
        assert worst[f] <= 1e-5, (f, worst[f])
    assert worst["epl"] <= 1e-4, worst["epl"]
    assert worst["epl_max"] > 0


@pytest.mark.parametrize("tile", [3, 4])
def test_fp32_warp_strips_many_strips_and_segments_against_oracle(P, tile):
    """The FP32 warp-strip 2D sweep on a grid of 6 full strips (28 columns)
    plus a ragged one and several 64- or 32-row segments, against the FP64
    oracle through first yield: stress within 1e-5, plastic strain within
    1e-4."""
    s = E.config(1, n=(180, 150), L=(1.0, 150 / 180), inclusion_radius=0.05)
    worst = run_fp32_vs_oracle(P, s, 6, kernel=(P.KERNEL_FUSED, tile))
    for f in ("txx", "tyy", "txy", "p"):
        assert worst[f] <= 1e-5, (f, worst[f])
    assert worst["epl"] <= 1e-4, worst["epl"]
    assert worst["epl_max"] > 0


@pytest.mark.parametrize("nd,prec", [(2, "fp64"), (3, "fp32")])
def test_solve_in_chunks_equals_one_solve(P, nd, prec):
    """ep_solve_chunks(1) called until the solve is decided performs the same
    iterations as one ep_solve_increment: same check iteration, same frozen
    point, fields bit for bit; PENDING is returned while undecided and a new
    increment abandons an undecided solve."""
    if nd == 2:
        s = E.config(1, n=(40, 34), tol=1e-9)
    else:
        s = E.config(3, n=(20, 17, 14), inclusion_radius=0.2)
    precision = P.FP64 if prec == "fp64" else P.FP32_MIXED
    fields = FIELDS_2D if nd == 2 else FIELDS_3D
    nchk = 20 if nd == 2 else 100
    ga = gpu_grid(P, s, precision, n_chk=nchk, freeze_iter=200 if nd == 3 else 0)
    gb = gpu_grid(P, s, precision, n_chk=nchk, freeze_iter=200 if nd == 3 else 0)
    pending = 0
    for inc in range(1, 8):
        ga.apply_increment_rates(rates_of(s), s.dt)
        ia = ga.solve_increment()
        gb.apply_increment_rates(rates_of(s), s.dt)
        while True:
            ib = gb.solve_chunks(1)
            if ib["status"] != P.PENDING:
                break
            pending += 1
            assert ib["iters"] % nchk == 0
        assert ib["status"] == 0 and ib["iters"] == ia["iters"] and ib["frozen_at"] == ia["frozen_at"]
        for f in fields:
            assert np.array_equal(ga.get(f), gb.get(f)), (inc, f)
    assert pending > 0 and ia["n_plastic"] > 0
    # an undecided solve is abandoned by the next increment
    gb.apply_increment_rates(rates_of(s), s.dt)
    assert gb.solve_chunks(1)["status"] == P.PENDING
    ga.apply_increment_rates(rates_of(s), s.dt)
    gb.apply_increment_rates(rates_of(s), s.dt)
    ia, ib = ga.solve_increment(), gb.solve_increment()
    assert ia["iters"] == ib["iters"]
    ga.close()
    gb.close()


def test_advection_fp64_parity_2d(P):
    """Advection of the old stress (Eq. j1) on: every increment after the
    first transports tau_hat and p_hat with the last converged velocity.
    Same iterations and fields within 1e-10 of the oracle through first
    yield; one increment applied twice on the GPU side only (advected once)."""
    s = E.config(1, n=(40, 33), tol=1e-9)
    g = gpu_grid(P, s, P.FP64, advection=True)
    o = O.from_setup(s, advection=True)
    for inc in range(1, 11):
        g.apply_increment_rates(rates_of(s), s.dt)
        if inc == 6:
            g.apply_increment_rates(rates_of(s), s.dt)
        ig = g.solve_increment()
        o.apply_increment(rates_of(s), s.dt)
        io = o.solve_increment()
        assert ig["iters"] == io["iters"], (inc, ig["iters"], io["iters"])
        sc = group_scales(o, FIELDS_2D)
        for f in FIELDS_2D:
            e = rel_err(g.get(f), o.get(f), sc[f])
            assert e <= 1e-10, (inc, f, e)
    assert io["n_plastic"] > 0
    g.close()


def test_advection_survives_snapshot_and_restore(P):
    """An increment solved, restored from the checkpoint taken before it and
    solved again advects the restored history again: same iterations, same
    fields bit for bit."""
    s = E.config(1, n=(32, 28), tol=1e-9)
    g = gpu_grid(P, s, P.FP64, advection=True)
    for _ in range(6):
        g.apply_increment_rates(rates_of(s), s.dt)
        g.solve_increment()
    g.snapshot()
    g.apply_increment_rates(rates_of(s), s.dt)
    i1 = g.solve_increment()
    f1 = {f: g.get(f) for f in FIELDS_2D}
    g.restore()
    g.apply_increment_rates(rates_of(s), s.dt)
    i2 = g.solve_increment()
    assert i1["iters"] == i2["iters"]
    for f in FIELDS_2D:
        np.testing.assert_array_equal(g.get(f), f1[f], err_msg=f)
    g.close()


@pytest.mark.parametrize("variant", [0, 3])
def test_advection_fp64_parity_3d(P, variant):
    """Advection on in 3D (x-z pure shear) with the staged and the register
    sweeps: every history component incl. the three edge families."""
    s = E.config(3, n=(17, 13, 11), tol=1e-9, precision="fp64", inclusion_radius=0.2)
    run_pair_kernel(P, s, 7, variant, 4, advection=True)


def test_advection_fp32_mixed_within_stated_bounds_3d(P):
    s = E.config(3, n=(16, 15, 14), inclusion_radius=0.15)
    worst = run_fp32_vs_oracle(P, s, 7, advection=True)
    for f in ("txx", "tyy", "tzz", "txy", "txz", "tyz", "p"):
        assert worst[f] <= 1e-5, (f, worst[f])
    assert worst["epl"] <= 1e-4, worst["epl"]


def test_pressure_anomaly_fp64_parity_2d(P):
    """The paper's symmetry-study box (2:1, uniform G and c, De = 1e6, no
    Jaumann term) seeded by an initial circular pressure anomaly p = c/2,
    written into the history on both sides: the anomaly is out of equilibrium,
    so the first increments iterate; same iterations and fields within 1e-10
    through first yield."""
    s = E.anomaly_setup(n=(96, 48), tol=1e-10)
    g = gpu_grid(P, s, P.FP64, jaumann=False)
    o = O.from_setup(s, jaumann=False)
    p0 = s.initial_pressure()
    g.set("p", p0)
    o.set("p", p0)
    for inc in range(1, 9):
        g.apply_increment_rates(rates_of(s), s.dt)
        ig = g.solve_increment()
        o.apply_increment(rates_of(s), s.dt)
        io = o.solve_increment()
        assert ig["iters"] == io["iters"], (inc, ig["iters"], io["iters"])
        assert ig["n_plastic"] == io["n_plastic"], (inc, ig["n_plastic"], io["n_plastic"])
        sc = group_scales(o, FIELDS_2D)
        for f in FIELDS_2D:
            e = rel_err(g.get(f), o.get(f), sc[f])
            assert e <= 1e-10, (inc, f, e)
    assert io["n_plastic"] > 0
    g.close()


def test_not_converged_keeps_state_and_reports(P):
    s = E.config(1, n=(32, 32))
    g = gpu_grid(P, s, P.FP64, max_iter=200, n_chk=100, tol=1e-14)
    for _ in range(6):
        g.apply_increment(1.0, s.dt, P.LOAD_XY)
        info = g.solve_increment(raise_on_fail=False)
    assert info["status"] == 5 and info["iters"] == 200
    with pytest.raises(P.EPError):
        g.solve_increment()  # still open: hits max_iter again
    g.commit_increment()


def test_nan_in_the_history_is_reported_as_diverged_and_the_grid_recovers(P):
    """Failure injection on the host (no GPU fault): a NaN written into the old stress through ep_set_fields reaches
    the residual norms, the solve returns EP_ERR_DIVERGED without
    committing, and the handle stays usable: with the finite history restored
    from a device checkpoint, the increment solves as on a grid that never
    saw the NaN.  A NaN
    cohesion is refused on the host."""
    s = E.config(1, n=(32, 28))
    g = gpu_grid(P, s, P.FP64)
    ref = gpu_grid(P, s, P.FP64)
    for _ in range(4):
        for x in (g, ref):
            x.apply_increment(1.0, s.dt, P.LOAD_XY)
            x.solve_increment()
    g.snapshot()
    bad = g.get("txx").copy()
    bad[14, 16] = np.nan
    g.set("txx", bad)
    g.apply_increment(1.0, s.dt, P.LOAD_XY)
    info = g.solve_increment(raise_on_fail=False)
    assert info["status"] == 6, info            # EP_ERR_DIVERGED
    assert np.isnan(g.get("txx")[14, 16])       # nothing committed
    g.restore()                                 # the finite history back, the increment abandoned
    g.apply_increment(1.0, s.dt, P.LOAD_XY)
    ig = g.solve_increment()
    ref.apply_increment(1.0, s.dt, P.LOAD_XY)
    ir = ref.solve_increment()
    assert ig["iters"] == ir["iters"]
    for f in FIELDS_2D:
        assert np.array_equal(g.get(f), ref.get(f)), f
    coh = s.cohesion()
    coh.ravel()[5] = np.nan
    with pytest.raises(P.EPError, match="not finite"):
        g.set_material(s.K, s.G, s.mu_s, s.phi_deg, s.psi_deg, coh)
    g.close()
    ref.close()


def test_tma_wait_that_runs_out_ends_the_solve_with_timeout(P):
    """A bounded device wait made to run out (the TMA sweep's plane-copy
    waits given a bound of 8 cycles, far below a copy's latency): the
    kernel records the timeout, waits with its default bound for the copies
    it issued and returns; the solve ends with EP_ERR_TIMEOUT, and with the
    default bound back the same increment solves as on an untouched grid."""
    s = E.config(3, n=(20, 17, 14), inclusion_radius=0.2, tol=1e-9)
    g = gpu_grid(P, s, P.FP64)
    ref = gpu_grid(P, s, P.FP64)
    for x in (g, ref):
        x.set_kernel(P.KERNEL_FUSED_TMA, 0)
        for _ in range(4):
            x.apply_increment_rates(rates_of(s), s.dt)
            x.solve_increment()
    g.set_solver(tol=s.tol, wait_cycles=8)
    g.apply_increment_rates(rates_of(s), s.dt)
    info = g.solve_increment(raise_on_fail=False)
    assert info["status"] == 7, info            # EP_ERR_TIMEOUT
    g.set_solver(tol=s.tol)
    g.apply_increment_rates(rates_of(s), s.dt)
    ig = g.solve_increment()
    ref.apply_increment_rates(rates_of(s), s.dt)
    ir = ref.solve_increment()
    assert ig["iters"] == ir["iters"] and ir["n_plastic"] > 0
    for f in FIELDS_3D:
        assert np.array_equal(g.get(f), ref.get(f)), f
    g.close()
    ref.close()


def test_argument_and_state_errors(P):
    with pytest.raises(P.EPError):
        P.Grid(2, (0, 5))
    g = P.Grid(2, (8, 8))
    with pytest.raises(P.EPError):
        g.apply_increment(1.0, 1e-4)            # no material yet
    with pytest.raises(P.EPError):
        g.set_material(2.0, 1.0, math.inf, 30.0, 5.0, np.ones(64))   # psi != 0
    g.set_material(2.0, 1.0, math.inf, 30.0, 0.0, np.ones(64))
    with pytest.raises(P.EPError):
        g.solve_increment()                     # no open increment
    with pytest.raises(P.EPError):
        g.set_solver(n_chk=3)                   # odd cadence
    with pytest.raises(P.EPError):
        g.apply_increment(1.0, 1e-4, P.LOAD_XZ)  # x-z loading needs 3D


def test_resume_from_fields_is_bit_identical(P):
    s = E.config(1, n=(24, 24))
    a = gpu_grid(P, s, P.FP64)
    for _ in range(5):
        a.apply_increment(1.0, s.dt, P.LOAD_XY); a.solve_increment()
    hist = ("vx", "vy", "txx", "tyy", "txy", "p", "epl", "ux", "uy", "exx", "eyy", "exy")
    saved = {f: a.get(f) for f in hist}
    b = gpu_grid(P, s, P.FP64)
    for f, v in saved.items():
        b.set(f, v)
    for _ in range(2):
        a.apply_increment(1.0, s.dt, P.LOAD_XY); ia = a.solve_increment()
        b.apply_increment(1.0, s.dt, P.LOAD_XY); ib = b.solve_increment()
        assert ia["iters"] == ib["iters"]
    for f in hist:
        assert np.array_equal(a.get(f), b.get(f)), f


def test_torch_workspace_and_stream(P):
    """Device memory and the stream come from PyTorch; the solve runs in the
    library's kernels on that stream."""
    import torch
    s = E.config(1, n=(20, 18))
    nbytes = P.workspace_bytes(2, s.n, P.FP64)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    ptr = (ws.data_ptr() + 255) // 256 * 256
    st = torch.cuda.Stream()
    g = P.Grid(2, s.n, precision=P.FP64, stream=st.cuda_stream, workspace=ptr, workspace_size=nbytes)
    g.set_material(s.K, s.G, s.mu_s, s.phi_deg, s.psi_deg, s.cohesion())
    g.set_solver(tol=s.tol)
    o = O.from_setup(s)
    for _ in range(6):
        g.apply_increment(1.0, s.dt, P.LOAD_XY); g.solve_increment()
        o.apply_increment([1.0, -1.0], s.dt); o.solve_increment()
    assert rel_err(g.get("txx"), o.get("txx")) <= 1e-10
    assert rel_err(g.get("p"), o.get("p"), np.abs(o.get("txx")).max()) <= 1e-10
    g.close()
    del ws


def run_pair_kernel(P, s, increments, variant, kz, precision=None, tol_fields=1e-10, dt_scale=(1.0,), **solver):
    precision = P.FP64 if precision is None else precision
    g = gpu_grid(P, s, precision, **solver)
    g.set_kernel(variant, kz)
    o = O.from_setup(s, **solver)
    fields = FIELDS_3D
    for inc in range(1, increments + 1):
        dt = s.dt * dt_scale[inc % len(dt_scale)]
        g.apply_increment_rates(rates_of(s), dt)
        ig = g.solve_increment()
        o.apply_increment(rates_of(s), dt)
        io = o.solve_increment()
        assert ig["iters"] == io["iters"], (inc, ig["iters"], io["iters"])
        sc = group_scales(o, fields)
        for f in fields:
            e = rel_err(g.get(f), o.get(f), sc[f])
            assert e <= tol_fields, (inc, f, e)
    g.close()


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("n,kz", [((17, 13, 11), 4), ((40, 21, 24), 5), ((33, 9, 7), 64), ((70, 20, 30), 0)])
def test_fused_kernel_fp64_parity_3d(P, n, kz, variant):
    """The fused one-kernel sweeps (cp.async and TMA plane streaming),
    instantiated in FP64, against the oracle at 1e-10: several x tiles,
    ragged y tiles and z-chunk boundaries."""
    s = E.config(3, n=n, tol=1e-9, precision="fp64", inclusion_radius=0.15)
    run_pair_kernel(P, s, 7, variant, kz)


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_fused_kernel_fp64_parity_3d_changing_dt(P, variant):
    """Maxwell medium (eta_ve, K dt and the PT weights all depend on dt) with
    dt changing between increments: the captured chunk graph is reused
    across increments, so every sweep must read the scalars of the current
    increment."""
    s = E.config(3, n=(19, 15, 12), tol=1e-9, precision="fp64", inclusion_radius=0.2, mu_s=2e-3)
    run_pair_kernel(P, s, 6, variant, 5, dt_scale=(1.0, 0.5, 2.0))


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_fused_kernel_fp64_parity_3d_xy_plane(P, variant):
    s = E.config(3, n=(20, 18, 13), tol=1e-9, precision="fp64", load_plane="xy", inclusion_radius=0.2)
    run_pair_kernel(P, s, 7, variant, 6)


def test_fused_fp32_matches_staged_fp32(P):
    """FP32 fused and FP32 staged sweeps agree to FP32 rounding over a fixed
    number of iterations of a plastic increment."""
    s = E.config(3, n=(36, 30, 28), tol=1e-6, inclusion_radius=0.15)
    out = []
    for variant in (P.KERNEL_STAGED, P.KERNEL_FUSED, P.KERNEL_FUSED_TMA, P.KERNEL_FUSED_REG):
        g = gpu_grid(P, s, P.FP32_MIXED)
        g.set_kernel(variant, 8)
        for inc in range(1, 6):
            if inc == 5:
                g.set_solver(tol=0.0, max_iter=400, n_chk=100)
            g.apply_increment(1.0, s.dt, P.LOAD_XZ)
            info = g.solve_increment(raise_on_fail=False)
            if info["status"] != 0:
                g.commit_increment()
        out.append({f: g.get(f) for f in FIELDS_3D})
        g.close()
    for names in GROUPS.values():
        present = [f for f in names if f in FIELDS_3D]
        scale = max(max(np.abs(out[0][f]).max() for f in present), 1e-30)
        for f in present:
            for k in (1, 2, 3):
                assert np.abs(out[k][f] - out[0][f]).max() / scale <= 2e-5, (k, f)


def test_fused_check_iteration_matches_the_staged_check_fp32_3d(P):
    """The FP32 register sweep's check iteration (the stopping measures
    reduced inside the z-march, the check snapshots and centre scales
    written by it) against the staged check iteration of the staged FP32
    sweep: after 400 iterations of a plastic increment the measures of the
    last check agree to the FP32 rounding of the two iterates, a solve to
    tolerance takes the same number of check intervals, and a NaN in the
    history ends the solve as diverged."""
    s = E.config(3, n=(36, 30, 28), tol=1e-6, inclusion_radius=0.15)
    infos, iters = [], []
    for variant in (P.KERNEL_STAGED, P.KERNEL_FUSED_REG):
        g = gpu_grid(P, s, P.FP32_MIXED, n_chk=100)
        g.set_kernel(variant, 8)
        for _ in range(4):
            g.apply_increment(1.0, s.dt, P.LOAD_XZ)
            g.solve_increment()
        g.snapshot()
        g.set_solver(tol=0.0, max_iter=400, n_chk=100)
        g.apply_increment(1.0, s.dt, P.LOAD_XZ)
        infos.append(g.solve_increment(raise_on_fail=False))
        g.restore()
        g.set_solver(tol=s.tol, max_iter=400000, n_chk=100)
        g.apply_increment(1.0, s.dt, P.LOAD_XZ)
        done = g.solve_increment()
        assert done["n_plastic"] > 0          # a plastic increment
        iters.append(done["iters"])
        g.close()
    a, b = infos
    assert a["status"] == b["status"] == 5 and a["iters"] == b["iters"] == 400, (a, b)
    assert abs(a["max_sigma"] - b["max_sigma"]) <= 1e-4 * a["max_sigma"]
    for k in ("eps_mom", "eps_tau", "eps_p", "eps_rel", "max_r"):
        assert abs(a[k] - b[k]) <= 5e-2 * max(abs(a[k]), 1e-30), (k, a[k], b[k])
    assert abs(iters[0] - iters[1]) <= 100, iters
    # a NaN in the old stress reaches the fused check at the first iteration
    g = gpu_grid(P, s, P.FP32_MIXED, n_chk=100)
    g.set_kernel(P.KERNEL_FUSED_REG, 8)
    for _ in range(4):
        g.apply_increment(1.0, s.dt, P.LOAD_XZ)
        g.solve_increment()
    bad = g.get("txx").copy()
    bad[14, 15, 18] = np.nan
    g.set("txx", bad)
    g.apply_increment(1.0, s.dt, P.LOAD_XZ)
    info = g.solve_increment(raise_on_fail=False)
    assert info["status"] == 6 and info["iters"] == 0, info   # EP_ERR_DIVERGED at the first check
    g.close()


@pytest.mark.parametrize("tile,n", [(0, (70, 37)), (1, (70, 37)), (2, (70, 37)), (3, (70, 37)), (3, (30, 150)),
                                    (4, (70, 37))])
def test_fused2d_fp64_parity(P, tile, n):
    """The fused 2D kernels (a batch of one), in FP64, against the oracle:
    block tiles (0-2) and warp strips (3, 4) over several strips, segments
    and ragged edges."""
    s = E.config(1, n=n, tol=1e-10)
    g = gpu_grid(P, s, P.FP64)
    g.set_kernel(P.KERNEL_FUSED, tile)
    o = O.from_setup(s)
    for inc in range(1, 8):
        g.apply_increment(1.0, s.dt, P.LOAD_XY)
        o.apply_increment([1.0, -1.0], s.dt)
        ig, io = g.solve_increment(), o.solve_increment()
        assert ig["iters"] == io["iters"], inc
        sc = group_scales(o, FIELDS_2D)
        for f in FIELDS_2D:
            assert rel_err(g.get(f), o.get(f), sc[f]) <= 1e-10, (inc, f)


@pytest.mark.parametrize("tile", [3, 4])
def test_fused2d_strips_match_tiles_on_tall_grids(P, tile):
    """Warp strips over several segments (64 / 32 rows) against the block
    tile kernel, both FP64 on the GPU: same iterations, fields within 1e-10."""
    s = E.config(1, n=(60, 560), tol=1e-9, c0=6e-4, inclusion_radius=0.1)
    g0 = gpu_grid(P, s, P.FP64)
    g0.set_kernel(P.KERNEL_FUSED, 0)
    g1 = gpu_grid(P, s, P.FP64)
    g1.set_kernel(P.KERNEL_FUSED, tile)
    plastic = 0
    for inc in range(1, 3):
        g0.apply_increment(1.0, s.dt, P.LOAD_XY)
        g1.apply_increment(1.0, s.dt, P.LOAD_XY)
        i0, i1 = g0.solve_increment(), g1.solve_increment()
        assert i0["iters"] == i1["iters"], inc
        plastic += i0["n_plastic"] > 0
        for f in FIELDS_2D:
            assert rel_err(g1.get(f), g0.get(f)) <= 1e-10, (inc, f)
    assert plastic >= 1
    g0.close(); g1.close()


def _batch_setups():
    sizes = [(24, 24), (31, 17), (40, 40), (16, 33), (9, 50)]
    out = []
    for q, n in enumerate(sizes):
        out.append(E.Setup("b%d" % q, 2, n, phi_deg=22.0 + 3 * q, c0=1.2e-3 + 1e-4 * q, inclusion_radius=0.1,
                           inclusion_centre=(0.05 * q - 0.1, 0.02 * q, 0.0), seed=4000 + q, tol=1e-9))
    return out


@pytest.mark.parametrize("tile", [0, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_solo_bit_for_bit(P, prec, tile):
    """Every grid advanced inside a batch equals its own solo solve exactly
    (same kernel arithmetic, same iteration count), for uneven sizes and
    materials; FP64 instances also match the oracle."""
    pr = P.FP64 if prec == "fp64" else P.FP32_MIXED
    setups = _batch_setups()
    tol = 1e-9 if prec == "fp64" else 1e-6
    grids = []
    for s in setups:
        g = gpu_grid(P, s, pr, tol=tol, max_iter=400000)
        g.set_kernel(P.KERNEL_FUSED, tile)
        grids.append(g)
    batch = P.Batch(grids)
    batch.set_tile(tile)
    solos = []
    for s in setups:
        g = gpu_grid(P, s, pr, tol=tol, max_iter=400000)
        g.set_kernel(P.KERNEL_FUSED, tile)
        solos.append(g)
    oracles = [O.from_setup(s, tol=tol) for s in setups] if prec == "fp64" else None
    try:
        _batch_vs_solo(P, batch, grids, setups, solos, oracles)
    finally:
        batch.close()


def _batch_vs_solo(P, batch, grids, setups, solos, oracles):
    for inc in range(1, 7):
        batch.apply_increment(1.0, 1e-4)
        infos, st = batch.solve_increment()
        for q, (s, g) in enumerate(zip(setups, solos)):
            g.apply_increment(1.0, 1e-4, P.LOAD_XY)
            i1 = g.solve_increment()
            assert infos[q]["iters"] == i1["iters"], (inc, q)
            for f in FIELDS_2D:
                assert np.array_equal(grids[q].get(f), g.get(f)), (inc, q, f)
            if oracles:
                o = oracles[q]
                o.apply_increment([1.0, -1.0], 1e-4)
                io = o.solve_increment()
                assert io["iters"] == i1["iters"], (inc, q)
                sc = group_scales(o, FIELDS_2D)
                for f in FIELDS_2D:
                    assert rel_err(g.get(f), o.get(f), sc[f]) <= 1e-10, (inc, q, f)


def test_batch_autotune_picks_a_tile_and_keeps_results(P):
    setups = _batch_setups()
    grids = [gpu_grid(P, s, P.FP32_MIXED, tol=1e-6) for s in setups]
    for g in grids:
        g.set_kernel(P.KERNEL_FUSED, 0)
    batch = P.Batch(grids)
    try:
        for inc in range(1, 6):
            batch.apply_increment(1.0, 1e-4)
            if inc == 5:
                tile = batch.autotune(5)
                assert tile in (0, 1, 2, 3, 4)
            infos, st = batch.solve_increment()
            assert st == 0
    finally:
        batch.close()


def run_frozen_pair(P, s, increments, variant=None, kz=0, freeze_iter=100, batch=False, tile=None):
    """GPU FP64 against the oracle with frozen plasticity (Sec. 3.3) forced
    early: same iterations, same freeze check, fields within 1e-10."""
    g = gpu_grid(P, s, P.FP64, freeze_iter=freeze_iter, freeze_eps=0.0)
    if variant is not None:
        g.set_kernel(variant, kz)
    if tile is not None:
        g.set_kernel(P.KERNEL_FUSED, tile)
    o = O.from_setup(s)
    o.set_freeze(freeze_iter, 0.0)
    B = P.Batch([g]) if batch else None
    if B is not None and tile is not None:
        B.set_tile(tile)
    try:
        return _frozen_loop(P, s, g, o, B, increments)
    finally:
        if B is not None:
            B.close()
        g.close()


def _frozen_loop(P, s, g, o, B, increments):
    batch = B is not None
    fields = FIELDS_2D if s.ndim == 2 else FIELDS_3D
    froze = 0
    for inc in range(1, increments + 1):
        if batch:
            B.apply_increment(s.a, s.dt)
            ig = B.solve_increment()[0][0]
        else:
            g.apply_increment_rates(rates_of(s), s.dt)
            ig = g.solve_increment()
        o.apply_increment(rates_of(s), s.dt)
        io = o.solve_increment()
        assert ig["iters"] == io["iters"], (inc, ig["iters"], io["iters"])
        assert ig["frozen_at"] == io["frozen_at"], (inc, ig["frozen_at"], io["frozen_at"])
        assert ig["n_plastic"] == io["n_plastic"], inc
        froze += io["frozen_at"] >= 0
        sc = group_scales(o, fields)
        for f in fields:
            e = rel_err(g.get(f), o.get(f), sc[f])
            assert e <= 1e-10, (inc, f, e)
    return froze


def test_frozen_plasticity_fp64_parity_2d_staged(P):
    s = E.config(1, n=(40, 36), tol=1e-9, inclusion_radius=0.12)
    assert run_frozen_pair(P, s, 9, variant=P.KERNEL_STAGED) >= 1


@pytest.mark.parametrize("tile", [0, 3])
def test_frozen_plasticity_fp64_parity_2d_batched(P, tile):
    s = E.config(1, n=(40, 36), tol=1e-9, inclusion_radius=0.12)
    assert run_frozen_pair(P, s, 9, batch=True, tile=tile) >= 1


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_frozen_plasticity_fp64_parity_3d(P, variant):
    s = E.config(3, n=(20, 17, 14), tol=1e-9, precision="fp64", inclusion_radius=0.2)
    assert run_frozen_pair(P, s, 7, variant=variant, kz=5) >= 1


# ------------------------------------------------- incompressible (NEXT-3) --
@pytest.mark.parametrize("kernel", [("staged", 0), ("strips", 1)])
def test_incompressible_fp64_parity_2d(P, kernel):
    """The incompressible variant (Eq. A2ssP2 in place of Eq. A2ssP: the
    pressure is pseudo-time state stepped by -K~ div v, starting at the old
    pressure; reading R9) against the oracle's: same iterations and fields
    within 1e-10 through first yield of an inclusion, with the staged sweep
    and with the fused warp strips."""
    s = E.config(1, n=(40, 33), tol=1e-9)
    g = gpu_grid(P, s, P.FP64, incompressible=True)
    if kernel[1]:
        g.set_kernel(P.KERNEL_FUSED, 3)
    else:
        g.set_kernel(P.KERNEL_STAGED, -1)
    o = O.from_setup(s, incompressible=True)
    for inc in range(1, 9):
        g.apply_increment_rates(rates_of(s), s.dt)
        ig = g.solve_increment()
        o.apply_increment(rates_of(s), s.dt)
        io = o.solve_increment()
        assert ig["iters"] == io["iters"], (inc, ig["iters"], io["iters"])
        sc = group_scales(o, FIELDS_2D)
        for f in FIELDS_2D:
            e = rel_err(g.get(f), o.get(f), sc[f])
            assert e <= 1e-10, (inc, f, e)
    assert io["n_plastic"] > 0
    g.close()


@pytest.mark.parametrize("variant", [0, 3])
def test_incompressible_fp64_parity_3d(P, variant):
    """The same in 3D (x-z pure shear) with the staged sweep and the register
    z-march kernel."""
    s = E.config(3, n=(17, 13, 11), inclusion_radius=0.25, tol=1e-9)
    g = gpu_grid(P, s, P.FP64, incompressible=True)
    g.set_kernel(variant, 4 if variant else -1)
    o = O.from_setup(s, incompressible=True)
    for inc in range(1, 7):
        g.apply_increment_rates(rates_of(s), s.dt)
        ig = g.solve_increment()
        o.apply_increment(rates_of(s), s.dt)
        io = o.solve_increment()
        assert ig["iters"] == io["iters"], (inc, ig["iters"], io["iters"])
        sc = group_scales(o, FIELDS_3D)
        for f in FIELDS_3D:
            e = rel_err(g.get(f), o.get(f), sc[f])
            assert e <= 1e-10, (inc, f, e)
    assert io["n_plastic"] > 0
    g.close()


def test_incompressible_fp32_within_stated_bounds_3d(P):
    """FP32 sweeps of the incompressible variant against the FP64 oracle:
    stress within 1e-5 and plastic strain within 1e-4."""
    s = E.config(3, n=(16, 15, 14), inclusion_radius=0.2)
    worst = run_fp32_vs_oracle(P, s, 7, incompressible=True)
    for f in ("txx", "tyy", "tzz", "txy", "txz", "tyz", "p"):
        assert worst[f] <= 1e-5, (f, worst[f])
    assert worst["epl"] <= 1e-4, worst["epl"]
    assert worst["epl_max"] > 0


# ------------------------------------- per-cell shear modulus (NEXT-2) -----
def _gaussian_with_noise(nd, n, **kw):
    """The heterogeneous box with +-1 % seeded cohesion noise: the box alone is
    mirror-symmetric, so rounding would decide which of several cells with
    equal stress yields first; the noise makes first yield one cell's."""
    s = E.gaussian_setup(nd, n=n, **kw)
    c = s.cohesion()
    u = E.uniform01(s.seed + 17, c.size).reshape(c.shape)
    s.extra["cohesion"] = c * (1.0 + 0.01 * (2.0 * u - 1.0))
    return s


@pytest.mark.parametrize("nd,mu_s", [(2, math.inf), (2, 2e-3), (3, math.inf)])
def test_per_cell_shear_modulus_fp64_parity(P, nd, mu_s):
    """The paper's heterogeneous box (Sec. 4.1: Gaussian G-bar and c-bar with
    the wall jump, plus seeded noise; reading R10 for where a per-cell G
    enters) against the
    oracle with the same per-cell modulus: same iterations and fields within
    1e-10 through first yield, in the elastic limit and with a Maxwell
    viscosity (which makes the weight c2 of the rotated old stress vary from
    point to point)."""
    n = (40, 33) if nd == 2 else (16, 13, 11)
    s = _gaussian_with_noise(nd, n, mu_s=mu_s, tol=1e-9)
    g = gpu_grid(P, s, P.FP64)
    g.set_shear_modulus(s.shear_modulus())
    o = O.from_setup(s)
    o.set_shear_modulus(s.shear_modulus())
    fields = FIELDS_2D if nd == 2 else FIELDS_3D
    for inc in range(1, 12 if nd == 2 else 14):
        g.apply_increment_rates(rates_of(s), s.dt)
        ig = g.solve_increment()
        o.apply_increment(rates_of(s), s.dt)
        io = o.solve_increment()
        assert ig["iters"] == io["iters"], (inc, ig["iters"], io["iters"])
        sc = group_scales(o, fields)
        for f in fields:
            e = rel_err(g.get(f), o.get(f), sc[f])
            assert e <= 1e-10, (inc, f, e)
    assert io["n_plastic"] > 0
    g.close()


def test_per_cell_shear_modulus_fp32_within_stated_bounds(P):
    """FP32 sweeps on the heterogeneous 2D box against the FP64 oracle:
    stress within 1e-5, plastic strain within 1e-4."""
    s = _gaussian_with_noise(2, (48, 40), tol=1e-6)
    g = gpu_grid(P, s, P.FP32_MIXED, tol=1e-6, max_iter=400000)
    g.set_shear_modulus(s.shear_modulus())
    o = O.from_setup(s, tol=1e-10)
    o.set_shear_modulus(s.shear_modulus())
    worst = {}
    for inc in range(1, 11):
        g.apply_increment_rates(rates_of(s), s.dt)
        g.solve_increment()
        o.apply_increment(rates_of(s), s.dt)
        o.solve_increment()
        sc = group_scales(o, FIELDS_2D)
        for f in FIELDS_2D:
            worst[f] = max(worst.get(f, 0.0), rel_err(g.get(f), o.get(f), sc[f]))
    for f in ("txx", "tyy", "txy", "p"):
        assert worst[f] <= 1e-5, (f, worst[f])
    assert worst["epl"] <= 1e-4 and o.get("epl").max() > 0, worst["epl"]
    g.close()
