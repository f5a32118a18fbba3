"""Pins of the numpy network oracle: its convolution against scipy's
correlation, and its layer table against a hand count of the parameters."""
import numpy as np
import pytest

from oracle import unet_oracle as U


def test_conv_matches_scipy_correlate_2d_and_3d():
    sig = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(3)
    for nd, shape in ((2, (6, 7)), (3, (4, 5, 6))):
        x = rng.normal(size=(2, 3) + shape)
        w = rng.normal(size=(4, 3, 27 if nd == 3 else 9))
        b = rng.normal(size=4)
        y = U.conv(x, w, b, 3)
        for n in range(2):
            for co in range(4):
                ref = b[co] + sum(sig.correlate(x[n, ci], w[co, ci].reshape((3,) * nd), mode="same")
                                  for ci in range(3))
                np.testing.assert_allclose(y[n, co], ref, rtol=1e-12, atol=1e-12)


def test_layer_table_counts():
    table, n = U.layer_table(2, 4, 2, 32, 3)
    taps = 9
    expect = (4 * 32 + 32 * 32 + 32 * 64 + 64 * 64 + 64 * 128 + 128 * 128 + 192 * 64 + 64 * 64 + 96 * 32 + 32 * 32) * taps
    expect += 32 * 2 + (32 + 32 + 64 + 64 + 128 + 128 + 64 + 64 + 32 + 32 + 2)
    assert n == expect and len(table) == 11


def test_pool_up_are_adjoint_up_to_scale():
    rng = np.random.default_rng(1)
    a = rng.normal(size=(1, 2, 8, 6))
    b = rng.normal(size=(1, 2, 4, 3))
    # <pool(a), b> = <a, up(b)> / 4 in 2D
    assert np.isclose((U.pool(a) * b).sum(), (a * U.up(b)).sum() / 4)


def test_fd_gradient_of_a_quadratic_is_exact():
    """The finite-difference gradient of the loss matches the closed form of
    its derivative with respect to the head biases (the loss is quadratic in
    them)."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 3, 4, 4))
    t = rng.normal(size=(2, 2, 4, 4))
    table, n = U.layer_table(2, 3, 2, 3, 1)
    p = rng.normal(size=n) * 0.3
    g = U.fd_gradient(p, x, t, 2, 3, 2, 3, 1)
    bo = table[-1][4]
    y = U.forward(p, x, 2, 3, 2, 3, 1)
    # dL/db_c = 2 sum_{n,y,x} (y - t)[n, c] / numel = 2 mean_c(y - t) / C
    analytic = 2 * (y - t).mean(axis=(0, 2, 3)) / y.shape[1]
    np.testing.assert_allclose(g[bo:bo + 2], analytic, rtol=1e-6)


def test_bf16_rounding_is_nearest_even():
    """round_bf16 keeps 8 significant bits, rounding to nearest with ties to
    even (the conversion the tensor-core forward applies to its inputs)."""
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5, 1.0 + 2.0 ** -7 + 2.0 ** -12])
    y = U.round_bf16(x)
    np.testing.assert_array_equal(y, [1.0, 1.0, 1.0 + 2.0 ** -6, 1.0, -2.5, 1.0 + 2.0 ** -7])
