"""Plain numpy definition of the warm-start network's features and targets.

TEST INFRASTRUCTURE: only the tests may import this module; the product
computes the same tensors in its own kernels.

Grids: cell arrays in numpy order ([z,] y, x).  The network's grid is made of
coarse cells, each the mean of the f^D fine cells it covers that lie inside
the grid (cells of the padding hold zero), padded to a multiple of 4 coarse
cells per side.

Scales, with |a| the largest loading rate, L_max the longest box side:
    S_v = 0.1 |a| L_max,  S_t = 2 G |a| dt,  S_e = 10 |a| dt.

Features of increment n (read before it starts), per fine cell:
    (v_{n-1} - v_{n-2}) mean of the two faces of the cell, / S_v  (nd)
    tau_hat normal / c                                             (nd)
    tau_hat shear, mean of the 4 vertices/edges around the cell, / c (ns)
    p_hat / c, 1 - s, c / max c, eps_pl / S_e                      (4)
Target of increment n (read after it is solved):
    (v_n - v_{n-1}) mean of the two faces / S_v                    (nd)
    (tau_n - tau_phys) normal / S_t                                (nd)
    (tau_n - tau_phys) shear, mean of the 4 around the cell, / S_t (ns)
where tau_n is the converged stress state and tau_phys the physical response
of the converged velocity with the old history.
"""
import numpy as np


def padded_dims(n, f=1):
    p = [((x + f - 1) // f + 3) // 4 * 4 for x in n]
    return tuple(p + [1] * (3 - len(p)))


def scales(rates, L, dt, G):
    a = max(abs(r) for r in rates) or 1.0
    return 0.1 * a * max(L), 2.0 * G * a * dt, 10.0 * a * dt


def _cells(a, ndim):
    a = np.asarray(a, np.float64)
    return a if ndim == 3 else a.reshape((1,) + a.shape[-2:])


def _centre_mean_faces(v, d, n):
    """mean of face component d over the two faces of every cell (3D order)."""
    ndim = len(n)
    a = _cells(v, ndim)
    ax = 2 - d
    lo = np.take(a, np.arange(n[d]), axis=ax)
    hi = np.take(a, np.arange(1, n[d] + 1), axis=ax)
    return 0.5 * (lo + hi)


def _shear_to_centre(t, c, ndim):
    """mean of shear component c over the 4 points around each cell."""
    a = _cells(t, ndim)
    axes = [2, 1] if ndim == 2 or c == 0 else ([2, 0] if c == 1 else [1, 0])
    for ax in axes:
        a = 0.5 * (np.take(a, np.arange(a.shape[ax] - 1), axis=ax) + np.take(a, np.arange(1, a.shape[ax]), axis=ax))
    return a


def pool(chans, n, f):
    """Coarse-cell means of fine cell channels (list of (nz, ny, nx) arrays),
    padded: array (channels, Zc, Yc, Xc)."""
    ndim = len(n)
    Xc, Yc, Zc = padded_dims(n, f)
    nz = n[2] if ndim == 3 else 1
    out = np.zeros((len(chans), Zc, Yc, Xc), dtype=np.float64)
    fz = f if ndim == 3 else 1
    for K in range((nz + fz - 1) // fz):
        for J in range((n[1] + f - 1) // f):
            for I in range((n[0] + f - 1) // f):
                sl = (slice(K * fz, min((K + 1) * fz, nz)), slice(J * f, min((J + 1) * f, n[1])),
                      slice(I * f, min((I + 1) * f, n[0])))
                for q, ch in enumerate(chans):
                    out[q, K, J, I] = ch[sl].mean()
    return out


def features(n, f, v_prev, v_prev2, tn, ts, p, scale, coh, epl, rates, L, dt, G):
    """Features (flat float32 array) of the next increment."""
    ndim = len(n)
    S_v, _, S_e = scales(rates, L, dt, G)
    c = _cells(coh, ndim)
    ic = np.where(c > 0, 1.0 / np.where(c > 0, c, 1.0), 0.0)
    chans = []
    for d in range(ndim):
        chans.append((_centre_mean_faces(v_prev[d], d, n) - _centre_mean_faces(v_prev2[d], d, n)) / S_v)
    for d in range(ndim):
        chans.append(_cells(tn[d], ndim) * ic)
    for k in range(len(ts)):
        chans.append(_shear_to_centre(ts[k], k, ndim) * ic)
    chans.append(_cells(p, ndim) * ic)
    chans.append(1.0 - _cells(scale, ndim))
    cm = np.abs(c).max()
    chans.append(c / (cm if cm > 0 else 1.0))
    chans.append(_cells(epl, ndim) / S_e)
    return pool(chans, n, f).astype(np.float32).reshape(-1)


def target(n, f, v_new, v_prev, tn_new, ts_new, tn_phys, ts_phys, rates, L, dt, G):
    """Target (flat float32 array) of the increment just solved."""
    ndim = len(n)
    S_v, S_t, _ = scales(rates, L, dt, G)
    chans = []
    for d in range(ndim):
        chans.append((_centre_mean_faces(v_new[d], d, n) - _centre_mean_faces(v_prev[d], d, n)) / S_v)
    for d in range(ndim):
        chans.append((_cells(tn_new[d], ndim) - _cells(tn_phys[d], ndim)) / S_t)
    for k in range(len(ts_new)):
        chans.append((_shear_to_centre(ts_new[k], k, ndim) - _shear_to_centre(ts_phys[k], k, ndim)) / S_t)
    return pool(chans, n, f).astype(np.float32).reshape(-1)
