"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only draws numbers: cohesion fields with a weak inclusion and
white noise, per-instance material draws for batches, and the named workload
presets.  It holds none of the solver's arithmetic, so both sides can take
their inputs from it without sharing any of the method.

Random numbers come from one counter-based generator: the i-th output of
splitmix64 started from ``seed`` (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), mapped to a double in [0, 1)
from its top 53 bits.  Draw i is a pure function of (seed, i), so every array
is reproducible element by element.

The workloads stand in for the paper's setups (a box under pure shear with a
weak seed, Sec. 4.1): the paper used no dataset, so every input here is
synthetic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of splitmix64 seeded with ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of :func:`splitmix64`."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def cell_centres(n, L):
    """Cell-centre coordinates per axis on the centred box [-L/2, L/2]."""
    return [(-0.5 * L[d] + (np.arange(n[d]) + 0.5) * (L[d] / n[d])) for d in range(len(n))]


def cohesion_field(n, L, c0, noise=0.01, seed=0, inclusion_radius=0.0,
                   inclusion_centre=None, inclusion_factor=0.5):
    """Per-cell cohesion c = c0 (1 + noise (2U - 1)), halved in a weak inclusion.

    ``n`` and ``L`` have 2 or 3 entries.  The array is returned in C order with
    x fastest, i.e. shape (ny, nx) or (nz, ny, nx); cell (i, j[, k]) draws
    U number i + nx (j + ny k).  A cell belongs to the inclusion when its centre
    lies within ``inclusion_radius`` of ``inclusion_centre`` (centre-sampled).
    """
    ndim = len(n)
    count = int(np.prod(n))
    u = uniform01(seed, count).reshape(tuple(reversed(n)))
    c = c0 * (1.0 + noise * (2.0 * u - 1.0))
    if inclusion_radius > 0.0:
        centre = inclusion_centre if inclusion_centre is not None else [0.0] * ndim
        axes = cell_centres(n, L)
        grids = np.meshgrid(*reversed(axes), indexing="ij")  # (z,)y,x order
        r2 = np.zeros_like(c)
        for d in range(ndim):
            r2 += (grids[ndim - 1 - d] - centre[d]) ** 2
        c = np.where(r2 <= inclusion_radius ** 2, inclusion_factor * c, c)
    return np.ascontiguousarray(c, dtype=np.float64)


@dataclass
class Setup:
    """One solve: grid, material, loading and solver settings."""
    name: str
    ndim: int
    n: tuple
    L: tuple = (1.0, 1.0, 1.0)
    K: float = 2.0
    G: float = 1.0
    mu_s: float = math.inf
    phi_deg: float = 30.0
    psi_deg: float = 0.0
    c0: float = 1.5e-3
    inclusion_radius: float = 0.05
    inclusion_centre: tuple = (0.0, 0.0, 0.0)
    noise: float = 0.01
    seed: int = 0
    a: float = 1.0
    dt: float = 1e-4
    load_plane: str = "xy"
    increments: int = 30
    tol: float = 1e-8
    precision: str = "fp64"
    extra: dict = field(default_factory=dict)

    def cohesion(self) -> np.ndarray:
        if "cohesion" in self.extra:
            return self.extra["cohesion"].copy()
        return cohesion_field(self.n, self.L[: self.ndim], self.c0, self.noise, self.seed,
                              self.inclusion_radius, self.inclusion_centre[: self.ndim])

    def shear_modulus(self):
        """The per-cell shear modulus of the setup, or None (uniform G)."""
        g = self.extra.get("shear_modulus")
        return None if g is None else g.copy()

    def initial_pressure(self):
        """The initial (history) pressure of the setup, or None (zero)."""
        a = self.extra.get("pressure_anomaly")
        if a is None:
            return None
        return pressure_anomaly(self.n, self.L[: self.ndim], a["value"], a["radius"])


def pressure_anomaly(n, L, value, radius, centre=None):
    """Initial pressure: ``value`` at cells whose centre lies within ``radius``
    of ``centre`` (default the box centre), 0 elsewhere; shape as
    :func:`cohesion_field`."""
    ndim = len(n)
    centre = centre if centre is not None else [0.0] * ndim
    axes = cell_centres(n, L)
    grids = np.meshgrid(*reversed(axes), indexing="ij")
    r2 = np.zeros(tuple(reversed(n)))
    for d in range(ndim):
        r2 += (grids[ndim - 1 - d] - centre[d]) ** 2
    return np.ascontiguousarray(np.where(r2 <= radius ** 2, value, 0.0), dtype=np.float64)


def anomaly_setup(n=(383, 191), **overrides) -> Setup:
    """The box of the paper's symmetry study (Sec. 4.3, "Symmetry versus
    non-symmetry"): a 2:1 plane-strain box, uniform G = 1 and cohesion
    c = 0.2e-2 G (no noise, no inclusion), Deborah number 1e6 (mu_s = 1e6 G t,
    the elastic limit), no Jaumann term, and a circular pressure anomaly
    p = c / 2 at the centre.  The paper prints no anomaly radius; 0.05 L_y is
    used.  Solver settings go in ``extra`` (``jaumann``)."""
    c = 2e-3
    s = Setup("2d-anomaly", 2, tuple(n), L=(2.0, 1.0, 1.0), mu_s=1e6, c0=c, inclusion_radius=0.0, noise=0.0,
              seed=6000, increments=180, tol=1e-10)
    s.extra = {"pressure_anomaly": {"value": 0.5 * c, "radius": 0.05}, "jaumann": False}
    for k, v in overrides.items():
        setattr(s, k, v)
    return s


def config(index: int, **overrides) -> Setup:
    """The five named workloads (seeds: index * 1000 + instance).

    1: 2D plane-strain elasto-plastic 64x64, 30 increments, tol 1e-8.
    2: 2D visco-elasto-plastic 511x511, eta/(G dt) = 10, 200 increments.
    3: 3D elasto-plastic 127^3 (oracle at 63^3), x-z pure shear, 100 increments.
    4: batch of 256 uneven 2D instances (see :func:`batch_setups`).
    5: 3D elasto-plastic 511^3, x-z pure shear, 60 increments, tol 1e-6.
    """
    if index == 1:
        s = Setup("2d-64-ep", 2, (64, 64), seed=1000, increments=30, tol=1e-8)
    elif index == 2:
        s = Setup("2d-511-vep", 2, (511, 511), mu_s=1e-3, seed=2000, increments=200, tol=1e-8)
    elif index == 3:
        s = Setup("3d-127-ep", 3, (127, 127, 127), seed=3000, load_plane="xz",
                  increments=100, tol=1e-6, precision="fp32")
    elif index == 5:
        s = Setup("3d-511-ep", 3, (511, 511, 511), seed=5000, load_plane="xz",
                  increments=60, tol=1e-6, precision="fp32")
    else:
        raise ValueError("config %d has no single-grid setup; use batch_setups()" % index)
    for k, v in overrides.items():
        setattr(s, k, v)
    return s


BATCH_SIZES = (127, 255, 383, 511)


def batch_setups(count: int = 256, base_seed: int = 4000, sizes=BATCH_SIZES) -> list:
    """Instances of the uneven 2D batch: n, phi, c0 and the inclusion drawn per instance.

    Instance b uses seed base_seed + b.  Its first five draws pick
    n ~ U{sizes}, phi ~ U[20, 35] deg, c0 ~ U[1e-3, 2e-3] G, r ~ U[0.03, 0.08]
    and the inclusion centre ~ U[-0.5 + r, 0.5 - r]^2 (two draws); the cohesion
    noise uses the separate stream seeded with base_seed + b + 2^32.
    """
    out = []
    for b in range(count):
        seed = base_seed + b
        u = uniform01(seed, 6)
        n = sizes[min(int(u[0] * len(sizes)), len(sizes) - 1)]
        phi = 20.0 + 15.0 * u[1]
        c0 = 1e-3 + 1e-3 * u[2]
        r = 0.03 + 0.05 * u[3]
        cx = -0.5 + r + (1.0 - 2.0 * r) * u[4]
        cy = -0.5 + r + (1.0 - 2.0 * r) * u[5]
        s = Setup("batch-%d" % b, 2, (n, n), phi_deg=phi, c0=c0, inclusion_radius=r,
                  inclusion_centre=(cx, cy, 0.0), seed=seed + (1 << 32), increments=50,
                  tol=1e-6, precision="fp32")
        out.append(s)
    return out


def gaussian_fields(n, L, G0=1.0, c0=2e-3, width=0.2, wall_band=0.05):
    """The paper's heterogeneous setup (Sec. 4.1): a shear modulus rising as a
    Gaussian from G0 at the centre to 1.2 G0 at the walls,
        G = G0 (1.2 - 0.2 exp(-(r / w)^2)),
    and a cohesion rising the same way from c0 at the centre towards 1.5 c0,
        c = c0 (1.5 - 0.5 exp(-(r / w)^2)),
    with a jump to 2 c0 within ``wall_band`` of any wall; r is the distance of
    the cell centre from the box centre, w = ``width`` times the shortest box
    side.  Shapes as :func:`cohesion_field`."""
    ndim = len(n)
    axes = cell_centres(n, L)
    grids = np.meshgrid(*reversed(axes), indexing="ij")
    r2 = np.zeros(tuple(reversed(n)))
    near_wall = np.zeros(tuple(reversed(n)), dtype=bool)
    for d in range(ndim):
        xd = grids[ndim - 1 - d]
        r2 += xd ** 2
        near_wall |= np.abs(xd) >= 0.5 * L[d] - wall_band * min(L)
    w = width * min(L)
    bump = np.exp(-r2 / w ** 2)
    G = G0 * (1.2 - 0.2 * bump)
    c = np.where(near_wall, 2.0 * c0, c0 * (1.5 - 0.5 * bump))
    return np.ascontiguousarray(G), np.ascontiguousarray(c)


def gaussian_setup(ndim=2, n=None, **overrides) -> Setup:
    """The box of the paper's heterogeneous runs (Sec. 4.1; Sec. 4.4 uses it
    at 511^2): Gaussian G-bar (1 at the centre, 1.2 at the walls) and c-bar
    (0.2e-2 at the centre, a jump to 0.4e-2 near the walls), phi = 30 deg,
    zero initial stress.  The paper prints neither the Gaussian's width nor
    the band of the jump; :func:`gaussian_fields` fixes both."""
    n = tuple(n) if n is not None else ((511, 511) if ndim == 2 else (127, 127, 127))
    s = Setup("%dd-gaussian" % ndim, ndim, n, c0=2e-3, inclusion_radius=0.0, noise=0.0, seed=7000,
              load_plane="xy" if ndim == 2 else "xz", increments=30, tol=1e-8)
    G, c = gaussian_fields(n, (1.0,) * ndim)
    s.extra = {"shear_modulus": G, "cohesion": c}
    for k, v in overrides.items():
        setattr(s, k, v)
    return s
