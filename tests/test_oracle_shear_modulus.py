"""Pins of the oracle's per-cell shear modulus (the paper's heterogeneous
G-bar, Sec. 4.1).

Fixed by the mathematics: in 3D x-z pure shear a modulus that varies only
with y leaves the homogeneous strain field in equilibrium (every stress is a
function of y alone and sigma_yy = 0), so the solve converges at once and
each layer carries 2 G(y) eps, or its own yield plateau B c; and a smooth
G(x, y) manufactured solution converges at second order in the grid size.
"""
import math

import numpy as np
import pytest

import oracle as O

K = 2.0
PHI = 30.0
_s = math.sin(math.radians(PHI))
B3 = 6 * math.cos(math.radians(PHI)) / (math.sqrt(3) * (3 - _s))


def _layered(n, coh, G_of_y, **solver):
    o = O.Oracle(3, n)
    o.set_material(K, 1.0, math.inf, PHI, 0.0, np.full(tuple(reversed(n)), coh))
    kw = dict(tol=1e-12)
    kw.update(solver)
    o.set_solver(**kw)
    Gc = np.broadcast_to(G_of_y[None, :, None], tuple(reversed(n))).copy()
    o.set_shear_modulus(Gc)
    return o


def test_layered_modulus_keeps_the_homogeneous_strain_exactly():
    """G varying from layer to layer in y (not smoothly): converged at
    k = 0, txx = -tzz = 2 G(y) eps, tyy = p = shear stress = 0."""
    n = (6, 9, 5)
    G_of_y = np.array([1.0, 1.7, 0.6, 1.2, 2.5, 0.9, 1.1, 1.4, 0.8])
    o = _layered(n, 1.0, G_of_y)
    for inc in range(1, 4):
        o.apply_increment([1.0, 0.0, -1.0], 1e-4)
        assert o.solve_increment()["iters"] == 0
        eps = inc * 1e-4
        exp = np.broadcast_to((2 * G_of_y * eps)[None, :, None], (n[2], n[1], n[0]))
        np.testing.assert_allclose(o.get("txx"), exp, rtol=1e-12)
        np.testing.assert_allclose(o.get("tzz"), -exp, rtol=1e-12)
        for f in ("tyy", "p", "txy", "txz", "tyz"):
            assert np.abs(o.get(f)).max() < 1e-17, f


def test_layered_modulus_reaches_each_layers_plateau():
    """With yield: layer y is elastic until 2 G(y) eps reaches B c and then
    stays on the plateau sqrt(J2) = B c; stiffer layers yield first."""
    n = (5, 6, 4)
    G_of_y = np.array([0.8, 1.0, 1.3, 1.6, 2.0, 2.4])
    c = 1.5e-3
    o = _layered(n, c, G_of_y)
    for inc in range(1, 12):
        o.apply_increment([1.0, 0.0, -1.0], 1e-4)
        assert o.solve_increment()["iters"] == 0
        eps = inc * 1e-4
        sj = np.sqrt(0.5 * (o.get("txx") ** 2 + o.get("tyy") ** 2 + o.get("tzz") ** 2))
        # in x-z pure shear sqrt(J2) = 2 G eps while elastic (txx = -tzz)
        exp = np.minimum(2 * G_of_y * eps, B3 * c)
        np.testing.assert_allclose(sj, np.broadcast_to(exp[None, :, None], sj.shape), rtol=1e-12)


def test_uniform_array_equals_the_scalar_modulus():
    n = (7, 6, 5)
    runs = []
    for arr in (False, True):
        o = O.Oracle(3, n)
        coh = np.full(tuple(reversed(n)), 1.5e-3)
        coh[2:4, 2:4, 2:4] *= 0.5
        o.set_material(K, 1.3, math.inf, PHI, 0.0, coh)
        o.set_solver(tol=1e-10)
        if arr:
            o.set_shear_modulus(np.full(tuple(reversed(n)), 1.3))
        for _ in range(9):
            o.apply_increment([1.0, 0.0, -1.0], 1e-4)
            o.solve_increment()
        runs.append({f: o.get(f) for f in ("txx", "txy", "p", "epl", "vx")})
    for f in runs[0]:
        np.testing.assert_array_equal(runs[0][f], runs[1][f])


def _mms_variable_G_2d(nc):
    """Manufactured elastic solution with G(x, y) = 1 + 0.4 sin(pi x) cos(pi y)
    and body force f = -div sigma(v*) from the exact derivatives."""
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    dt = 1e-4
    Gxy = 1 + 0.4 * sp.sin(sp.pi * x) * sp.cos(sp.pi * y)
    vx = x + 0.3 * sp.cos(sp.pi * x) * sp.sin(sp.pi * y)
    vy = -y - 0.2 * sp.sin(sp.pi * x) * sp.cos(sp.pi * y)
    exx, eyy = sp.diff(vx, x), sp.diff(vy, y)
    exy = (sp.diff(vx, y) + sp.diff(vy, x)) / 2
    div = exx + eyy
    p = -K * dt * div
    txx = 2 * Gxy * dt * (exx - div / 3)
    tyy = 2 * Gxy * dt * (eyy - div / 3)
    txy = 2 * Gxy * dt * exy
    fx = -(sp.diff(txx - p, x) + sp.diff(txy, y))
    fy = -(sp.diff(tyy - p, y) + sp.diff(txy, x))
    lam = lambda e: sp.lambdify((x, y), e, "numpy")
    h = 1.0 / nc
    xf = -0.5 + np.arange(nc + 1) * h
    xc = -0.5 + (np.arange(nc) + 0.5) * h
    Xf, Yc = np.meshgrid(xf, xc)
    Xc, Yf = np.meshgrid(xc, xf)
    Xcc, Ycc = np.meshgrid(xc, xc)
    bx = np.broadcast_to(lam(fx)(Xf, Yc), Xf.shape)
    by = np.broadcast_to(lam(fy)(Xc, Yf), Xc.shape)
    return (lam(vx)(Xf, Yc), lam(vy)(Xc, Yf)), (bx, by), lam(Gxy)(Xcc, Ycc), dt


def test_manufactured_solution_with_variable_modulus_is_second_order():
    errs = []
    for nc in (16, 32, 64):
        (vxe, vye), (bx, by), Gc, dt = _mms_variable_G_2d(nc)
        o = O.Oracle(2, (nc, nc))
        o.set_material(K, 1.0, math.inf, PHI, 0.0, np.ones((nc, nc)))
        o.set_solver(tol=1e-12)
        o.set_shear_modulus(Gc)
        o.apply_increment([1.0, -1.0], dt, body_force=(bx, by))
        o.solve_increment()
        errs.append(max(np.abs(o.get("vx") - vxe).max(), np.abs(o.get("vy") - vye).max()))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(r > 1.8 for r in rates), (errs, rates)


def test_rejects_non_positive_moduli():
    o = O.Oracle(2, (4, 3))
    o.set_material(K, 1.0, math.inf, PHI, 0.0, np.ones((3, 4)))
    bad = np.ones((3, 4))
    bad[1, 2] = 0.0
    with pytest.raises(RuntimeError):
        o.set_shear_modulus(bad)
    with pytest.raises(ValueError):
        o.set_shear_modulus(np.ones(5))


def test_gaussian_setup_yields_at_the_centre_first():
    """The paper's heterogeneous box (Gaussian G-bar and c-bar): the first
    plastic cells sit in the weak centre, scales never exceed 1, the plastic
    strain never decreases."""
    import ep_inputs as E
    s = E.gaussian_setup(n=(24, 24), tol=1e-9)
    o = O.from_setup(s)
    o.set_shear_modulus(s.shear_modulus())
    epl_prev = np.zeros((24, 24))
    first = None
    for inc in range(1, 12):
        o.apply_increment([1.0, -1.0], s.dt)
        info = o.solve_increment()
        sc = o.get("scale")
        assert sc.max() <= 1.0
        epl = o.get("epl")
        assert (epl >= epl_prev).all()
        epl_prev = epl
        if info["n_plastic"] and first is None:
            first = inc
            j, i = np.nonzero(sc < 1)
            r = np.hypot((i + 0.5) / 24 - 0.5, (j + 0.5) / 24 - 0.5)
            assert r.max() < 0.2, r.max()
    assert first is not None
