"""Pins of the oracle's advection of the old stress (the v_k d sigma_ij / dx_k
term of the Jaumann rate, Eq. j1; explicit first-order upwind, once per
increment, with the previous increment's converged velocity).

Each pin is fixed by the mathematics of the transport equation, not by the
oracle: at Courant number one, upwind transport is an exact one-cell shift;
on a linear field, upwind differences and linear interpolation of a linear
velocity are exact, so the step equals f - dt v(x).grad f of the continuous
equation; with Courant number below one the scheme is a convex combination,
so it keeps the field's bounds and its constants; and a homogeneous stress
is not changed by transport at all.
"""
import math

import numpy as np
import pytest

import ep_inputs as E
import oracle as O

# staggering per dimension (1: on grid lines, 0: at centres) of each field
STAG = {"txx": (0, 0, 0), "tyy": (0, 0, 0), "tzz": (0, 0, 0), "p": (0, 0, 0),
        "txy": (1, 1, 0), "txz": (1, 0, 1), "tyz": (0, 1, 1),
        "vx": (1, 0, 0), "vy": (0, 1, 0), "vz": (0, 0, 1)}
HIST = {2: ["txx", "tyy", "p", "txy"], 3: ["txx", "tyy", "tzz", "p", "txy", "txz", "tyz"]}


def _coords(ndim, n, L, name):
    """Coordinates (x, y[, z]) of the points of a field, arrays in (z,) y, x order."""
    st = STAG[name]
    ext = [n[d] + st[d] for d in range(ndim)]
    if ndim == 2 and name in ("txy",):
        ext = [n[0] + 1, n[1] + 1]
    axes = [-0.5 * L[d] + (np.arange(ext[d]) + (0.0 if st[d] else 0.5)) * L[d] / n[d] for d in range(ndim)]
    grids = np.meshgrid(*reversed(axes), indexing="ij")    # (z,) y, x
    return list(reversed(grids))                             # x, y[, z]


def _walls(ndim, n, name, shape):
    """Mask of free-slip wall points of a shear field (none for centre fields)."""
    st = STAG[name]
    m = np.zeros(shape, dtype=bool)
    for d in range(ndim):
        if st[d] and name.startswith("t") and name not in ("txx", "tyy", "tzz"):
            ax = ndim - 1 - d
            idx = [slice(None)] * ndim
            idx[ax] = 0; m[tuple(idx)] = True
            idx[ax] = -1; m[tuple(idx)] = True
    return m


def _grid(ndim, n, L):
    return O.Oracle(ndim, n, L)


def _set_velocity(o, ndim, n, L, fn):
    """Face velocities v_e = fn(e, x_e) at each face point."""
    for e, name in enumerate(["vx", "vy", "vz"][:ndim]):
        xs = _coords(ndim, n, L, name)
        o.set(name, fn(e, xs[e]))


@pytest.mark.parametrize("ndim,axis,sign", [(2, 0, 1), (2, 0, -1), (2, 1, 1), (2, 1, -1),
                                            (3, 0, 1), (3, 1, -1), (3, 2, 1), (3, 2, -1)])
def test_courant_one_is_an_exact_shift(ndim, axis, sign):
    """|v| dt = h: every point takes its upwind neighbour's value exactly; the
    inflow layer (no upwind neighbour) keeps its value; wall points of the
    shear fields stay zero."""
    n = (16, 8) if ndim == 2 else (6, 5, 7)
    L = tuple(x / 16 for x in n)          # h = 1/16 in every dimension
    dt, U = 1.0 / 64, 4.0 * sign          # U dt = 1/16 = h
    o = _grid(ndim, n, L)
    _set_velocity(o, ndim, n, L, lambda e, x: np.full(x.shape, U if e == axis else 0.0))
    rng = np.random.default_rng(7 + ndim * 10 + axis)
    old = {}
    for name in HIST[ndim]:
        shape = o.get(name).shape
        f = rng.integers(-50, 51, size=shape).astype(np.float64)
        f[_walls(ndim, n, name, shape)] = 0.0
        o.set(name, f)
        old[name] = f
    o.advect(dt)
    ax = ndim - 1 - axis
    for name, f in old.items():
        exp = f.copy()
        src = [slice(None)] * ndim
        dst = [slice(None)] * ndim
        if sign > 0:
            dst[ax], src[ax] = slice(1, None), slice(0, -1)
        else:
            dst[ax], src[ax] = slice(0, -1), slice(1, None)
        exp[tuple(dst)] = f[tuple(src)]
        w = _walls(ndim, n, name, f.shape)
        exp[w] = f[w]
        np.testing.assert_array_equal(o.get(name), exp, err_msg=name)


@pytest.mark.parametrize("ndim", [2, 3])
def test_linear_field_follows_the_continuous_transport(ndim):
    """Diagonal velocity gradient v_e = r_e x_e and a linear field
    f = g . x: the step equals f - dt sum_e r_e x_e g_e wherever the upwind
    neighbour exists (every component's interpolation to every staggering is
    exercised, incl. the 8-point mean of v_z at xy-edges); at an inflow wall
    the normal term drops (zero gradient)."""
    n = (12, 10) if ndim == 2 else (8, 7, 6)
    L = (1.0, 0.9, 0.8)[:ndim]
    r = (1.0, -0.7) if ndim == 2 else (1.0, 0.6, -1.3)
    gr = (0.3, -1.1) if ndim == 2 else (0.3, -1.1, 0.7)
    dt = 1e-3
    o = _grid(ndim, n, L)
    _set_velocity(o, ndim, n, L, lambda e, x: r[e] * x)
    for name in HIST[ndim]:
        xs = _coords(ndim, n, L, name)
        o.set(name, sum(gr[e] * xs[e] for e in range(ndim)))
    o.advect(dt)
    for name in HIST[ndim]:
        xs = _coords(ndim, n, L, name)
        f = sum(gr[e] * xs[e] for e in range(ndim))
        exp = f.copy()
        for e in range(ndim):
            v = r[e] * xs[e]
            ax = ndim - 1 - e
            q = np.indices(f.shape)[ax]
            has_up = np.where(v > 0, q >= 1, q <= f.shape[ax] - 2)
            exp -= dt * np.where(has_up & (v != 0), v * gr[e], 0.0)
        w = _walls(ndim, n, name, f.shape)
        exp[w] = f[w]
        np.testing.assert_allclose(o.get(name), exp, rtol=0, atol=1e-14, err_msg=name)


@pytest.mark.parametrize("ndim", [2, 3])
def test_bounds_and_constants_are_kept(ndim):
    """Courant number below one: each new value is a convex combination of
    old values, so no new extremum appears; a constant field is unchanged."""
    n = (14, 11) if ndim == 2 else (7, 6, 8)
    L = (1.0, 1.0, 1.0)[:ndim]
    rng = np.random.default_rng(3)
    o = _grid(ndim, n, L)
    r = (1.0, -1.0, 0.5)
    _set_velocity(o, ndim, n, L, lambda e, x: r[e] * x + 0.2 * rng.standard_normal(x.shape))
    old = {}
    for name in HIST[ndim]:
        shape = o.get(name).shape
        f = rng.random(shape)
        f[_walls(ndim, n, name, shape)] = 0.0
        o.set(name, f)
        old[name] = f
    o.advect(0.01)     # max |v| dt / h ~ 0.1 per dimension
    for name, f in old.items():
        g = o.get(name)
        assert g.min() >= f.min() - 1e-15 and g.max() <= f.max() + 1e-15, name
        assert np.abs(g - f).max() > 0, name
    for name in HIST[ndim]:
        shape = o.get(name).shape
        c = np.full(shape, 0.37)
        w = _walls(ndim, n, name, shape)
        c[w] = 0.0
        o.set(name, c)
    o.advect(0.01)
    for name in ("txx", "p"):
        np.testing.assert_array_equal(o.get(name), 0.37)


@pytest.mark.parametrize("ndim", [2, 3])
def test_homogeneous_elastic_closed_form_holds_with_advection(ndim):
    """A homogeneous stress is not changed by transport: the P1 closed form
    (txx = -tyy (or -tzz) = 2 G eps, p = 0) holds with advection on."""
    n = (10, 8) if ndim == 2 else (6, 5, 7)
    o = O.Oracle(ndim, n)
    o.set_material(2.0, 1.0, math.inf, 30.0, 0.0, np.ones(tuple(reversed(n))))
    o.set_solver(tol=1e-12, advection=True)
    rates = [1.0, -1.0] if ndim == 2 else [1.0, 0.0, -1.0]
    for inc in range(1, 4):
        o.apply_increment(rates, 1e-4)
        assert o.solve_increment()["iters"] == 0
        np.testing.assert_allclose(o.get("txx"), 2e-4 * inc, rtol=1e-12)
        np.testing.assert_allclose(o.get("tzz" if ndim == 3 else "tyy"), -2e-4 * inc, rtol=1e-12)
        assert np.abs(o.get("p")).max() < 1e-17


def test_advection_acts_once_per_committed_increment():
    """Nothing to advect before the first commit; applying an increment twice
    advects once; and with a heterogeneous stress the term does change the
    solution from the second increment on."""
    s = E.config(1, n=(20, 18), tol=1e-10)

    def run(advection, reapply):
        o = O.from_setup(s, advection=advection)
        out = []
        for inc in range(1, 9):
            o.apply_increment([1.0, -1.0], s.dt)
            if reapply and inc == 8:
                o.apply_increment([1.0, -1.0], s.dt)
            o.solve_increment()
            out.append(o.get("txx").copy())
        return out

    off, on, twice = run(False, False), run(True, False), run(True, True)
    np.testing.assert_array_equal(on[0], off[0])
    for a, b in zip(on, twice):
        np.testing.assert_array_equal(a, b)
    assert np.abs(on[-1] - off[-1]).max() > 1e-12
