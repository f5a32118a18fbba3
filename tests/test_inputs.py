"""The seeded input generators that both the oracle and the CUDA path read.

splitmix64 is pinned to its published outputs (Steele, Lea and Flood,
OOPSLA 2014; the reference implementation's sequences for seeds 0 and
1234567), and each field generator to a brute-force loop over cells.
"""
import math

import numpy as np
import pytest

import ep_inputs as E


def test_splitmix64_published_sequences():
    assert [int(x) for x in E.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(x) for x in E.splitmix64(1234567, 2)] == [6457827717110365317, 3203168211198807973]
    # draw i depends on (seed, i) only
    assert int(E.splitmix64(1234567, 1, offset=1)[0]) == 3203168211198807973


def test_uniform01_range_and_mean():
    u = E.uniform01(42, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3


def test_cohesion_field_by_brute_force():
    n, L = (9, 7), (1.0, 0.8)
    c = E.cohesion_field(n, L, 1.5e-3, noise=0.01, seed=5, inclusion_radius=0.2, inclusion_centre=(0.1, -0.05))
    u = E.uniform01(5, n[0] * n[1])
    for j in range(n[1]):
        for i in range(n[0]):
            x = -0.5 * L[0] + (i + 0.5) * L[0] / n[0]
            y = -0.5 * L[1] + (j + 0.5) * L[1] / n[1]
            v = 1.5e-3 * (1.0 + 0.01 * (2.0 * u[i + n[0] * j] - 1.0))
            if (x - 0.1) ** 2 + (y + 0.05) ** 2 <= 0.2 ** 2:
                v *= 0.5
            assert c[j, i] == v


def test_pressure_anomaly_by_brute_force():
    s = E.anomaly_setup(n=(40, 20))
    p = s.initial_pressure()
    assert p.shape == (20, 40)
    dx, dy = 2.0 / 40, 1.0 / 20
    for j in range(20):
        for i in range(40):
            x, y = -1.0 + (i + 0.5) * dx, -0.5 + (j + 0.5) * dy
            inside = x * x + y * y <= 0.05 ** 2
            assert p[j, i] == (1e-3 if inside else 0.0)
    # the symmetry study's box: uniform cohesion, no noise, no Jaumann term
    c = s.cohesion()
    assert np.all(c == 2e-3)
    assert s.extra["jaumann"] is False and s.mu_s == 1e6 and s.L[:2] == (2.0, 1.0)
    big = E.anomaly_setup().initial_pressure()
    assert big.shape == (191, 383) and np.array_equal(big, big[::-1, ::-1])
    assert (big > 0).sum() == sum(1 for j in range(191) for i in range(383)
                                  if (-1.0 + (i + 0.5) * 2 / 383) ** 2 + (-0.5 + (j + 0.5) / 191) ** 2 <= 0.0025)
    assert math.isclose(big.max(), 1e-3)


def test_gaussian_fields_by_brute_force():
    n, L = (12, 11), (1.0, 1.0)          # no cell centre on the edge of the wall band
    G, c = E.gaussian_fields(n, L)
    w = 0.2
    for j in range(n[1]):
        for i in range(n[0]):
            x, y = -0.5 + (i + 0.5) / n[0], -0.5 + (j + 0.5) / n[1]
            bump = math.exp(-(x * x + y * y) / w ** 2)
            assert G[j, i] == pytest.approx(1.0 * (1.2 - 0.2 * bump), rel=1e-14)
            wall = abs(x) >= 0.45 or abs(y) >= 0.45
            assert c[j, i] == pytest.approx(4e-3 if wall else 2e-3 * (1.5 - 0.5 * bump), rel=1e-14)
    s = E.gaussian_setup(n=(16, 16))
    assert s.shear_modulus().shape == (16, 16) and s.cohesion().shape == (16, 16)
    assert s.shear_modulus().min() > 1.0 and s.shear_modulus().max() < 1.2
