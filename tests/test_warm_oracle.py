"""Pins of the numpy definition of the warm-start features and targets.

A velocity change linear in x has cell-centre means equal to its value at
the centres, so the velocity channel is that line over its largest face
value; the exact extrapolation v_n = 2 v_{n-1} - v_{n-2} has a zero target
(the network's correction to "repeat the last increment"); the padding
outside the grid is zero.
"""
import numpy as np

from oracle import warm_oracle as W


def _faces_2d(n, fx, fy):
    nx, ny = n
    xf = -0.5 + np.arange(nx + 1) / nx
    yc = -0.5 + (np.arange(ny) + 0.5) / ny
    xc = -0.5 + (np.arange(nx) + 0.5) / nx
    yf = -0.5 + np.arange(ny + 1) / ny
    Xf, Yc = np.meshgrid(xf, yc)
    Xc, Yf = np.meshgrid(xc, yf)
    return [fx(Xf, Yc), fy(Xc, Yf)]


def test_linear_change_gives_the_centre_values_over_the_largest_face_value():
    n = (10, 7)
    v2 = _faces_2d(n, lambda x, y: 0 * x, lambda x, y: 0 * y)
    v1 = _faces_2d(n, lambda x, y: 0.3 * x, lambda x, y: -0.1 * y)
    scale = np.full((7, 10), 0.75)
    coh = np.linspace(1.0, 2.0, 70).reshape(7, 10)
    f, S = W.features(n, v1, v2, scale, coh)
    assert S == np.float64(0.15)          # 0.3 * 0.5 at the x walls
    f = f.reshape(4, 1, 8, 12)
    xc = -0.5 + (np.arange(10) + 0.5) / 10
    yc = -0.5 + (np.arange(7) + 0.5) / 7
    np.testing.assert_allclose(f[0, 0, :7, :10], np.broadcast_to(0.3 * xc / 0.15, (7, 10)), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(f[1, 0, :7, :10], np.broadcast_to((-0.1 * yc / 0.15)[:, None], (7, 10)), atol=1e-7)
    np.testing.assert_allclose(f[2, 0, :7, :10], 0.25)
    np.testing.assert_allclose(f[3, 0, :7, :10], coh / 2.0, rtol=1e-7)
    assert not f[:, :, 7:, :].any() and not f[:, :, :, 10:].any()


def test_exact_extrapolation_has_a_zero_target():
    rng = np.random.default_rng(1)
    n = (6, 5, 4)
    shapes = [(4, 5, 7), (4, 6, 6), (5, 5, 6)]
    v2 = [rng.random(s) for s in shapes]
    v1 = [rng.random(s) for s in shapes]
    v0 = [2 * a - b for a, b in zip(v1, v2)]
    f, S = W.features(n, v1, v2, rng.random((4, 5, 6)), rng.random((4, 5, 6)) + 0.5)
    t = W.target(n, v0, v1, S, f)
    assert np.abs(t).max() < 1e-6
    assert t.size == 3 * 8 * 8 * 4
