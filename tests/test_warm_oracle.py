"""Pins of the numpy definition of the warm-start features and targets
(oracle/warm_oracle.py), from what the definition fixes by construction:
centre means of linear fields are their centre values, the mean of the 4
vertices/edges of a linear field is its centre value, coarse cells average
the fine cells inside the grid (ragged ones included), padding is zero, and a
converged state equal to the physical response with no velocity change has a
zero target.
"""
import numpy as np

from oracle import warm_oracle as W

G, DT, RATES, L2 = 1.0, 1e-4, (1.0, -1.0), (1.0, 0.8)
S_V, S_T, S_E = 0.1 * 1.0 * 1.0, 2.0 * 1.0 * 1.0 * 1e-4, 10.0 * 1e-4


def _coords(n, L):
    """centre and node coordinates per dimension."""
    c = [-0.5 * L[d] + (np.arange(n[d]) + 0.5) * L[d] / n[d] for d in range(len(n))]
    f = [-0.5 * L[d] + np.arange(n[d] + 1) * L[d] / n[d] for d in range(len(n))]
    return c, f


def _fields_2d(n, L, fx, fy, fs):
    (xc, yc), (xf, yf) = _coords(n, L)
    vx = fx(*np.meshgrid(xf, yc))          # (ny, nx + 1)
    vy = fy(*np.meshgrid(xc, yf))          # (ny + 1, nx)
    txy = fs(*np.meshgrid(xf, yf))         # (ny + 1, nx + 1)
    return vx, vy, txy


def test_linear_fields_give_their_centre_values():
    n = (10, 7)
    zero = _fields_2d(n, L2, lambda x, y: 0 * x, lambda x, y: 0 * y, lambda x, y: 0 * x)
    v1 = _fields_2d(n, L2, lambda x, y: 0.03 * x + 0.01, lambda x, y: -0.02 * y, lambda x, y: 2e-4 * x - 1e-4 * y)
    (xc, yc), _ = _coords(n, L2)
    X, Y = np.meshgrid(xc, yc)
    coh = 1e-3 + 1e-4 * X
    tn = [3e-4 * X, -2e-4 * Y]
    p = 5e-4 + 1e-4 * Y
    scale = np.full(n[::-1], 0.75)
    epl = np.full(n[::-1], 2e-3)
    f = W.features(n, 1, [v1[0], v1[1]], [zero[0], zero[1]], tn, [v1[2]], p, scale, coh, epl, RATES, L2, DT, G)
    f = f.reshape(9, 1, 8, 12).astype(np.float64)
    sl = (0, slice(0, 7), slice(0, 10))
    np.testing.assert_allclose(f[0][sl], (0.03 * X + 0.01) / S_V, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(f[1][sl], -0.02 * Y / S_V, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(f[2][sl], tn[0] / coh, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(f[3][sl], tn[1] / coh, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(f[4][sl], (2e-4 * X - 1e-4 * Y) / coh, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(f[5][sl], p / coh, rtol=1e-6)
    np.testing.assert_allclose(f[6][sl], 0.25)
    np.testing.assert_allclose(f[7][sl], coh / coh.max(), rtol=1e-6)
    np.testing.assert_allclose(f[8][sl], 2.0, rtol=1e-6)
    assert not f[:, :, 7:, :].any() and not f[:, :, :, 10:].any()


def test_coarse_cells_average_the_fine_cells_inside_the_grid():
    n = (7, 5, 6)     # f = 2: ragged coarse cells in x and y
    rng = np.random.default_rng(3)
    sh = (6, 5, 7)
    chans = [rng.random(sh) for _ in range(2)]
    out = W.pool(chans, n, 2)
    assert out.shape == (2, 4, 4, 4)   # ceil(6/2), ceil(5/2), ceil(7/2) padded to 4
    for q in range(2):
        assert np.isclose(out[q, 0, 0, 0], chans[q][0:2, 0:2, 0:2].mean())
        assert np.isclose(out[q, 1, 2, 3], chans[q][2:4, 4:5, 6:7].mean())   # ragged corner: 2 x 1 x 1 cells
        assert np.isclose(out[q, 2, 1, 2], chans[q][4:6, 2:4, 4:6].mean())
        assert out[q, 3].sum() == 0.0                                     # padding
    # a constant pools to itself at every coarse cell that covers the grid
    c = W.pool([np.full(sh, 0.7)], n, 3)
    assert np.allclose(c[0, :2, :2, :3], 0.7) and c[0, 2:].sum() == 0 and c[0, :, 2:].sum() == 0


def test_3d_shear_means_of_linear_fields_and_zero_target():
    n = (4, 3, 5)
    L3 = (1.0, 0.75, 1.25)
    rng = np.random.default_rng(1)
    (xc, yc, zc), (xf, yf, zf) = _coords(n, L3)

    def grid(zs, ys, xs, fn):
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        return fn(X, Y, Z)

    lin = lambda X, Y, Z: 1e-4 * (1 + 2 * X - Y + 3 * Z)
    ts = [grid(zc, yf, xf, lin), grid(zf, yc, xf, lin), grid(zf, yf, xc, lin)]
    centre = grid(zc, yc, xc, lin)
    coh = np.full((5, 3, 4), 1e-3)
    v = [rng.random((5, 3, 5)), rng.random((5, 4, 4)), rng.random((6, 3, 4))]
    tn = [rng.random((5, 3, 4)) * 1e-3 for _ in range(3)]
    f = W.features(n, 1, v, v, tn, ts, np.zeros((5, 3, 4)), np.ones((5, 3, 4)), coh, np.zeros((5, 3, 4)),
                   (1.0, 0.0, -1.0), L3, DT, G).reshape(13, 8, 4, 4)
    for k in range(3):
        np.testing.assert_allclose(f[6 + k, :5, :3, :4], centre / 1e-3, rtol=1e-6)
    assert not f[:3].any()                 # no velocity change
    t = W.target(n, 1, v, v, tn, ts, tn, ts, (1.0, 0.0, -1.0), L3, DT, G)
    assert t.size == 9 * 8 * 4 * 4 and not t.any()
    # a uniform stress change over the increment: the target is that change / S_t
    t = W.target(n, 1, v, v, [a + 4e-4 for a in tn], ts, tn, ts, (1.0, 0.0, -1.0), L3, DT, G).reshape(9, 8, 4, 4)
    np.testing.assert_allclose(t[3:6, :5, :3, :4], 4e-4 / S_T, rtol=1e-6)
