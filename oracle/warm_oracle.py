"""Plain numpy definition of the warm-start network's features and targets.

TEST INFRASTRUCTURE: only the tests may import this module; the product
computes the same tensors in its own kernels.

An increment n's features are read before it starts, from the two last
converged velocities v_{n-1} and v_{n-2} (face arrays, walls included):
  S = max over all faces of |v_{n-1} - v_{n-2}|;
  channel d < ndim: the mean of (v_{n-1} - v_{n-2})_d over the two faces of
    each cell in direction d, divided by S (0 if S = 0);
  channel ndim: 1 - s, with s the last return scale of each cell;
  channel ndim + 1: c / max|c|;
laid out as (ndim + 2) channels over a box of Zp x Yp x Xp cells (x fastest;
each size rounded up to a multiple of 4), zero outside the grid.  The target
of increment n, read after it is solved, is the same centre mean of
v_n - v_{n-1} over the same S, minus the velocity channels of the features:
a network that outputs zero reproduces "repeat the last increment".
"""
import numpy as np


def padded_dims(n):
    p = [(x + 3) // 4 * 4 for x in n]
    return tuple(p + [1] * (3 - len(p)))


def _centre_means(dv, n, inv):
    """Per component, the cell-centre mean of a face field times inv, in
    (z, y, x) order (2D: one z layer)."""
    ndim = len(n)
    out = []
    for d in range(ndim):
        ax = ndim - 1 - d
        lo = np.take(dv[d], np.arange(n[d]), axis=ax)
        hi = np.take(dv[d], np.arange(1, n[d] + 1), axis=ax)
        c = 0.5 * (lo + hi) * inv
        out.append(c if ndim == 3 else c[None])
    return out


def features(n, v_prev, v_prev2, scale, coh):
    """(features as a flat float32 array, S) for grid size n, the last two
    converged face velocities (lists of arrays in the binding's shapes), the
    last return scales and the cohesion (cell arrays)."""
    ndim = len(n)
    dv = [np.asarray(a, np.float64) - np.asarray(b, np.float64) for a, b in zip(v_prev, v_prev2)]
    S = max(np.abs(x).max() for x in dv)
    inv = 1.0 / S if S > 0.0 else 0.0
    Xp, Yp, Zp = padded_dims(n)
    out = np.zeros((ndim + 2, Zp, Yp, Xp), dtype=np.float32)
    nz = n[2] if ndim == 3 else 1
    for d, c in enumerate(_centre_means(dv, n, inv)):
        out[d, :nz, :n[1], :n[0]] = c
    cells = lambda a: (np.asarray(a, np.float64) if ndim == 3 else np.asarray(a, np.float64)[None])
    out[ndim, :nz, :n[1], :n[0]] = 1.0 - cells(scale)
    cm = np.abs(np.asarray(coh)).max()
    out[ndim + 1, :nz, :n[1], :n[0]] = cells(coh) / (cm if cm > 0 else 1.0)
    return out.reshape(-1), S


def target(n, v_new, v_prev, S, feat):
    """Target of the increment solved from features `feat` (flat, as above)."""
    ndim = len(n)
    dv = [np.asarray(a, np.float64) - np.asarray(b, np.float64) for a, b in zip(v_new, v_prev)]
    inv = 1.0 / S if S > 0.0 else 0.0
    Xp, Yp, Zp = padded_dims(n)
    f = np.asarray(feat, np.float32).reshape(ndim + 2, Zp, Yp, Xp)
    out = np.zeros((ndim, Zp, Yp, Xp), dtype=np.float32)
    nz = n[2] if ndim == 3 else 1
    for d, c in enumerate(_centre_means(dv, n, inv)):
        out[d, :nz, :n[1], :n[0]] = c.astype(np.float32) - f[d, :nz, :n[1], :n[0]]
    return out.reshape(-1)
