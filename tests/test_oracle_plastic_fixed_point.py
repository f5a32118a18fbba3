"""Pins of the oracle's plastic return at vertices and edges (Sec. 3.3 with the
relaxed-trial reading, Eqs. A2ssP, A23ssP, A6-A6121lambda).

1. The converged plastic increments of the oracle equal the root of an
   independent numpy statement of the pseudo-steady fixed point
   (tests/fixed_point_numpy.py), found by Newton's method with a
   finite-difference Jacobian, on 2x2, 3x3, 4x3 (dx != dy), Maxwell, 2x2x2 and
   3x2x2 (dx, dy, dz all different) grids with several yielding centres.
2. The same comparison fails when a plausible slip is planted in a copy of the
   oracle: the minimum instead of the mean of the adjacent centre scales, or a
   wrong neighbour in an edge's set of centres.
3. An exact invariant of the return at every centre of a converged increment
   (P5): the centre's normal deviator and the shear averaged from its
   vertices/edges, each edge value divided by the mean scale of its centres
   and multiplied by the centre's own scale, lie on the yield surface where
   the centre yields and inside it elsewhere, to rounding (1e-12 Y_max).
"""
import math
import os

import numpy as np
import pytest

import ep_inputs as E
import oracle as O
from fixed_point_numpy import Problem

CN = {2: ["txx", "tyy"], 3: ["txx", "tyy", "tzz"]}
SH = {2: ["txy"], 3: ["txy", "txz", "tyz"]}


def _get(o, name):
    a = o.get(name)
    return a.reshape(a.shape[-2:]) if o.ndim == 2 else a


def _plastic_increment(nd, n, L, mu_s, incs, seed, lib_path=None):
    """Run the oracle to the start of increment `incs` on a grid with a
    +-30 % cohesion field and one weak centre; return the oracle, the inputs
    of that increment and its converged result."""
    rng = np.random.default_rng(seed)
    nc = int(np.prod(n))
    coh = 1.5e-3 * (1.0 + 0.3 * (2.0 * rng.random(nc) - 1.0))
    coh[nc // 2] *= 0.5
    o = O.Oracle(nd, n, L, lib_path=lib_path)
    o.set_material(2.0, 1.0, mu_s, 30.0, 0.0, coh)
    o.set_solver(tol=1e-13, n_chk=2, max_iter=4000000)
    rates = [1.0, -1.0] if nd == 2 else [1.0, 0.0, -1.0]
    dt = 1e-4
    for inc in range(1, incs + 1):
        o.apply_increment(rates, dt)
        if inc < incs:
            o.solve_increment()
    names = ["v0x", "v0y", "v0z"][:nd] + CN[nd] + SH[nd] + ["p", "coh"]
    hist = {k: _get(o, k) for k in names}
    bt = o.pt_params()[0]
    info = o.solve_increment()
    return o, hist, bt, info, dt


CASES = [
    (2, (2, 2), (1.0, 1.0), math.inf, 9),
    (2, (3, 3), (1.0, 1.0), math.inf, 9),
    (2, (4, 3), (1.0, 0.8), math.inf, 10),
    (2, (3, 3), (1.0, 1.0), 1e-3, 14),
    (3, (2, 2, 2), (1.0, 1.0, 1.0), math.inf, 11),
    (3, (3, 2, 2), (1.0, 0.9, 0.8), math.inf, 11),
]


def _compare(nd, n, L, mu_s, incs, lib_path=None):
    """Largest field difference (L-infinity, relative to each group's scale)
    between the oracle's converged increment and the Newton root, and the
    number of yielding centres."""
    o, hist, bt, info, dt = _plastic_increment(nd, n, L, mu_s, incs, seed=1, lib_path=lib_path)
    pr = Problem(nd, n, L, 2.0, 1.0, mu_s, 30.0, dt, bt, hist)
    x0 = pr.pack([hist["v0" + c] for c in "xyz"[:nd]], [hist[k] for k in CN[nd]], [hist[k] for k in SH[nd]],
                 hist["p"])
    x, _ = pr.solve(x0)
    v, tc, te, p = pr.unpack(x)
    _, s = pr.residual(x)
    sig = max(np.abs(_get(o, k)).max() for k in CN[nd] + SH[nd] + ["p"])
    err = 0.0
    for d, c in enumerate("xyz"[:nd]):
        ref = _get(o, "v" + c)
        err = max(err, np.abs(v[d] - ref).max() / np.abs(ref).max())
    for d, k in enumerate(CN[nd]):
        err = max(err, np.abs(tc[d] - _get(o, k)).max() / sig)
    for c, k in enumerate(SH[nd]):
        err = max(err, np.abs(te[c] - _get(o, k)).max() / sig)
    err = max(err, np.abs(p - _get(o, "p")).max() / sig)
    return err, int((s < 1).sum()), info


@pytest.mark.parametrize("nd,n,L,mu_s,incs", CASES)
def test_plastic_increment_equals_newton_root_of_the_fixed_point(nd, n, L, mu_s, incs):
    err, n_plastic_np, info = _compare(nd, n, L, mu_s, incs)
    nc = int(np.prod(n))
    assert info["n_plastic"] >= 2 and n_plastic_np == info["n_plastic"]
    if nc > 4:
        assert info["n_plastic"] < nc       # yielding and elastic centres side by side
    # the oracle stops at eps_res <= 1e-13; the root is exact to rounding
    assert err <= 1e-10, err


def _variant(tag, edit):
    src = O.source()
    new = edit(src)
    assert new != src
    return O.build_variant(new, tag)


def _min_for_mean(src):
    """vertex/edge scale: the minimum of the adjacent centre scales"""
    out = []
    for line in src.split("\n"):
        if "double sb = 0.25 * (" in line:
            inner = line.split("0.25 * (", 1)[1].rsplit(");", 1)[0]
            a, b, c, d = [t.strip() for t in inner.split(" + ")]
            line = line.split("double sb")[0] + "double sb = fmin(fmin(%s, %s), fmin(%s, %s));" % (a, b, c, d)
        out.append(line)
    return "\n".join(out)


def _wrong_edge_neighbour(src):
    """xz-edge scale: one of its four centres replaced by a neighbour at the
    other z-level (a wrong neighbour set)"""
    old = "double sb = 0.25 * (g->s[CI(i - 1, j, k - 1)] + g->s[CI(i, j, k - 1)]"
    assert old in src
    return src.replace(old, "double sb = 0.25 * (g->s[CI(i - 1, j, k)] + g->s[CI(i, j, k - 1)]")


@pytest.mark.parametrize("tag,edit,cases", [
    ("minmean", _min_for_mean, [CASES[1], CASES[4]]),
    ("edgeset", _wrong_edge_neighbour, [CASES[5]]),
])
def test_planted_return_slips_fail_the_fixed_point_pin(tag, edit, cases):
    path = _variant(tag, edit)
    try:
        for case in cases:
            err, _, _ = _compare(*case, lib_path=path)
            assert err > 1e-6, (tag, case, err)
    finally:
        os.remove(path)


def _edge_to_centre(a, nd, c):
    """mean of a shear component's 4 points around each centre"""
    axes = [(1, 0)] if nd == 2 else [(2, 1), (2, 0), (1, 0)]
    for ax in axes[c]:
        a = 0.5 * (np.take(a, range(a.shape[ax] - 1), axis=ax) + np.take(a, range(1, a.shape[ax]), axis=ax))
    return a


def _centres_to_edge(s, nd, c):
    """mean of the 4 centres around each interior point of a shear component
    (full array of the component, walls 0)"""
    axes = [(1, 0)] if nd == 2 else [(2, 1), (2, 0), (1, 0)]
    out_shape = list(s.shape)
    for ax in axes[c]:
        out_shape[ax] += 1
    m = s
    for ax in axes[c]:
        m = 0.5 * (np.take(m, range(m.shape[ax] - 1), axis=ax) + np.take(m, range(1, m.shape[ax]), axis=ax))
    full = np.zeros(out_shape)
    sl = [slice(None)] * s.ndim
    for ax in axes[c]:
        sl[ax] = slice(1, -1)
    full[tuple(sl)] = m
    return full


@pytest.mark.parametrize("nd", [2, 3])
def test_p5_centre_return_lies_on_the_yield_surface(nd):
    """P5 with the bound the return reading implies: at every centre of every
    converged increment, sqrt(J2) of (its normal deviator, s_c times the mean
    over its vertices/edges of tau_e / s_bar_e) equals Y = max(0, A p + B c)
    where it yields and does not exceed it elsewhere, to 1e-12 Y_max."""
    if nd == 2:
        s = E.config(1, n=(24, 20), increments=9)
        rates, A, B = [1.0, -1.0], 0.5, math.cos(math.radians(30.0))
    else:
        s = E.config(3, n=(10, 9, 8), inclusion_radius=0.25, increments=9)
        rates = [1.0, 0.0, -1.0]
        d = math.sqrt(3.0) * 2.5
        A, B = 3.0 / d, 6.0 * math.cos(math.radians(30.0)) / d
    o = O.from_setup(s, tol=1e-9)
    seen_plastic = 0
    for inc in range(1, 10):
        o.apply_increment(rates, s.dt)
        o.solve_increment()
        sc = _get(o, "scale")
        p, coh = _get(o, "p"), _get(o, "coh")
        Y = np.maximum(0.0, A * p + B * coh)
        J2 = sum(0.5 * _get(o, k) ** 2 for k in CN[nd])
        ok = np.ones_like(sc, dtype=bool)
        for c, k in enumerate(SH[nd]):
            sbar = _centres_to_edge(sc, nd, c)
            te = _get(o, k)
            T = np.divide(te, sbar, out=np.zeros_like(te), where=sbar > 0)
            # a centre next to an edge whose neighbours all sit at the apex
            # (s_bar = 0) has no recoverable trial there
            interior = np.zeros_like(te, dtype=bool)
            sl = [slice(None)] * te.ndim
            axes = [(1, 0)] if nd == 2 else [(2, 1), (2, 0), (1, 0)]
            for ax in axes[c]:
                sl[ax] = slice(1, -1)
            interior[tuple(sl)] = True
            bad = interior & (sbar <= 0)
            ok &= _edge_to_centre(bad.astype(float), nd, c) == 0
            J2 = J2 + (sc * _edge_to_centre(T, nd, c)) ** 2
        sj = np.sqrt(J2)
        tol = 1e-12 * Y.max()
        pl = (sc < 1) & ok
        el = (sc == 1) & ok
        assert np.abs(sj[pl] - Y[pl]).max(initial=0.0) <= tol
        assert (sj[el] - Y[el]).max(initial=-1.0) <= tol
        seen_plastic += int(pl.sum())
    assert seen_plastic > 0
