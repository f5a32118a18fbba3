"""Pins of the oracle's incompressible variant (Sec. 3.2: Eq. A2ssP2, the
pseudo-transient form of div v = 0, replaces the compressible pressure
equation A2ssP; all other equations are unchanged).

Fixed by the mathematics, not by the oracle: a homogeneous pure shear is
divergence-free, so it needs no pressure and keeps the elastic closed form;
the compressible solution tends to the incompressible one as K -> infinity,
with an error of order 1/K; the converged velocity is divergence-free
(recomputed here from the face velocities); and the plastic increments keep
the invariants of the compressible solver.
"""
import math

import numpy as np
import pytest

import ep_inputs as E
import oracle as O

PHI = 30.0
A2, B2 = math.sin(math.radians(PHI)), math.cos(math.radians(PHI))


@pytest.mark.parametrize("ndim", [2, 3])
def test_homogeneous_pure_shear_keeps_the_elastic_closed_form(ndim):
    n = (10, 8) if ndim == 2 else (6, 5, 7)
    o = O.Oracle(ndim, n)
    o.set_material(2.0, 1.0, math.inf, PHI, 0.0, np.ones(tuple(reversed(n))))
    o.set_solver(tol=1e-12, incompressible=True)
    rates = [1.0, -1.0] if ndim == 2 else [1.0, 0.0, -1.0]
    for inc in range(1, 4):
        o.apply_increment(rates, 1e-4)
        assert o.solve_increment()["iters"] == 0
        np.testing.assert_allclose(o.get("txx"), 2e-4 * inc, rtol=1e-12)
        np.testing.assert_allclose(o.get("tzz" if ndim == 3 else "tyy"), -2e-4 * inc, rtol=1e-12)
        assert np.abs(o.get("p")).max() < 1e-18


def _anomaly(ndim, n, incompressible, K=2.0):
    """Elastic box with an initial pressure anomaly (out of equilibrium)."""
    L = (2.0, 1.0, 1.0)[:ndim]
    s = E.Setup("inc", ndim, n, L=L + (1.0,) * (3 - ndim), K=K, mu_s=1e6, c0=1.0, inclusion_radius=0.0,
                noise=0.0, tol=1e-12, load_plane="xz" if ndim == 3 else "xy")
    o = O.from_setup(s, jaumann=False, incompressible=incompressible, max_iter=2000000)
    o.set("p", E.pressure_anomaly(n, L, 1e-3, 0.2))
    rates = [1.0, -1.0] if ndim == 2 else [1.0, 0.0, -1.0]
    o.apply_increment(rates, s.dt)
    info = o.solve_increment()
    names = ["txx", "tyy", "txy", "p", "vx", "vy"] + (["tzz", "txz", "tyz", "vz"] if ndim == 3 else [])
    return info, {f: o.get(f) for f in names}, L


def _dist(a, b):
    """Largest difference, each field relative to its group's largest value
    (velocities, stresses)."""
    out = 0.0
    for f in a:
        grp = [g for g in a if (g[0] == "v") == (f[0] == "v")]
        out = max(out, np.abs(a[f] - b[f]).max() / max(np.abs(a[g]).max() for g in grp))
    return out


@pytest.mark.parametrize("ndim,n", [(2, (32, 16)), (3, (12, 8, 7))])
def test_compressible_solution_tends_to_the_incompressible_one(ndim, n):
    """K -> infinity: the distance to the incompressible answer falls by a
    factor 10 per decade of K (first order in 1/K)."""
    _, inc, _ = _anomaly(ndim, n, True)
    d = [_dist(inc, _anomaly(ndim, n, False, K=K)[1]) for K in (1e2, 1e3, 1e4)]
    assert 8.0 < d[0] / d[1] < 12.0 and 8.0 < d[1] / d[2] < 12.0, d
    assert d[2] < 5e-3, d


@pytest.mark.parametrize("ndim,n", [(2, (32, 16)), (3, (12, 8, 7))])
def test_converged_velocity_is_divergence_free(ndim, n):
    info, f, L = _anomaly(ndim, n, True)
    assert info["iters"] > 0
    h = [L[d] / n[d] for d in range(ndim)]
    div = (f["vx"][..., 1:] - f["vx"][..., :-1]) / h[0]
    if ndim == 2:
        div = div + (f["vy"][1:, :] - f["vy"][:-1, :]) / h[1]
    else:
        div = div + (f["vy"][:, 1:, :] - f["vy"][:, :-1, :]) / h[1] + (f["vz"][1:] - f["vz"][:-1]) / h[2]
    # strain rates are of order a = 1
    assert np.abs(div).max() <= 1e-10
    # and the compressible solver does not give that (the anomaly relaxes)
    _, fc, _ = _anomaly(ndim, n, False)
    divc = (fc["vx"][..., 1:] - fc["vx"][..., :-1]) / h[0]
    assert np.abs(divc).max() > 1e-6


def test_plastic_increments_keep_the_invariants():
    """Incompressible inclusion run into yield: scales never above 1, the
    plastic strain never decreases, the centre deviator stays on or inside
    the yield surface (with the same allowance for the averaged vertex shear
    as the compressible pin), and yielding starts in the weak inclusion."""
    s = E.config(1, n=(32, 32), increments=9)
    o = O.from_setup(s, tol=1e-9, incompressible=True)
    epl_prev = np.zeros((32, 32))
    first = None
    for inc in range(1, s.increments + 1):
        o.apply_increment([1.0, -1.0], s.dt)
        info = o.solve_increment()
        sc = o.get("scale")
        assert sc.max() <= 1.0
        epl = o.get("epl")
        assert (epl >= epl_prev).all()
        epl_prev = epl
        txx, tyy, txy, p = o.get("txx"), o.get("tyy"), o.get("txy"), o.get("p")
        txy_c = 0.25 * (txy[:-1, :-1] + txy[1:, :-1] + txy[:-1, 1:] + txy[1:, 1:])
        sj = np.sqrt(0.5 * (txx ** 2 + tyy ** 2) + txy_c ** 2)
        Y = np.maximum(0, A2 * p + B2 * o.get("coh"))
        assert (sj - Y).max() <= 0.05 * Y.max()
        if info["n_plastic"] and first is None:
            first = inc
            weak = o.get("coh") < 1e-3
            assert (sc[weak] < 1).any() and not (sc[~weak] < 1).all()
    assert first is not None
