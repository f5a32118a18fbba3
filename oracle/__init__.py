"""Python handle on the FP64 CPU oracle (``oracle/ep_oracle.c``).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2305_01701_gb300``) never imports it and shares no code with it.

The library is compiled from source with the host C compiler on first use
(``build()``), into ``oracle/lib/``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ep_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libeporacle.so")
_lock = threading.Lock()
_lib = None

# field ids (numbering matches the product library's public header)
FIELDS = ["vx", "vy", "vz", "txx", "tyy", "tzz", "txy", "txz", "tyz", "p", "epl",
          "ux", "uy", "uz", "exx", "eyy", "ezz", "exy", "exz", "eyz", "coh", "eii", "scale",
          "v0x", "v0y", "v0z", "rx", "ry", "rz"]
FIELD_ID = {n: i for i, n in enumerate(FIELDS)}

OK, ERR_ARG, ERR_OOM, ERR_STATE, ERR_NOT_CONVERGED, ERR_DIVERGED = 0, 1, 3, 4, 5, 6


class Info(C.Structure):
    _fields_ = [("iters", C.c_long), ("eps_res", C.c_double), ("eps_mom", C.c_double),
                ("eps_tau", C.c_double), ("eps_p", C.c_double), ("eps_rel", C.c_double),
                ("max_r", C.c_double), ("max_sigma", C.c_double), ("n_plastic", C.c_long),
                ("sxx_int_centre", C.c_double), ("sxx_int_right", C.c_double),
                ("status", C.c_int), ("frozen_at", C.c_long)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            os.makedirs(_LIBDIR, exist_ok=True)
            tmp = _LIB + ".%d.tmp" % os.getpid()
            cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
                   "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


_LIB_OMP = os.path.join(_LIBDIR, "ep_oracle_omp.so")


def build_omp(force: bool = False):
    """The same source compiled with -fopenmp (its per-element loops then run
    on several threads, with the same results bit for bit); returns the
    library's path, or None where the compiler has no OpenMP."""
    with _lock:
        if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
            os.makedirs(_LIBDIR, exist_ok=True)
            tmp = _LIB_OMP + ".%d.tmp" % os.getpid()
            cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE", "-fopenmp",
                   "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
            if subprocess.run(cmd, capture_output=True).returncode != 0:
                return None
            os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def threads(n: int = 0, path: str | None = None) -> int:
    """Set (n > 0) and return the thread count of the oracle library at
    `path` (default: the plain build, always 1)."""
    return int(lib(path).or_threads(int(n)))


def build_variant(source: str, tag: str) -> str:
    """Compile a modified copy of the oracle's source (a test that plants a
    mistake in the oracle to show that a pin catches it) into
    ``oracle/lib/variant_<tag>.so``; returns its path."""
    os.makedirs(_LIBDIR, exist_ok=True)
    src = os.path.join(_LIBDIR, "variant_%s_%d.c" % (tag, os.getpid()))
    out = os.path.join(_LIBDIR, "variant_%s_%d.so" % (tag, os.getpid()))
    with open(src, "w") as f:
        f.write(source)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                    "-o", out, src, "-lm"], check=True)
    os.remove(src)
    return out


def source() -> str:
    with open(_SRC) as f:
        return f.read()


_variants = {}


def lib(path: str | None = None):
    """The oracle library (or a variant built by build_variant)."""
    global _lib
    if path is not None:
        if path not in _variants:
            _variants[path] = _load(path)
        return _variants[path]
    if _lib is None:
        _lib = _load(build())
    return _lib


def _load(path):
    L = C.CDLL(path)
    P, D, I, Lg = C.c_void_p, C.c_double, C.c_int, C.c_long
    DP = C.POINTER(C.c_double)
    L.or_create.restype = P
    L.or_create.argtypes = [I, C.POINTER(C.c_int), DP]
    L.or_destroy.argtypes = [P]
    L.or_set_material.argtypes = [P, D, D, D, D, D, DP]
    L.or_set_solver.argtypes = [P, D, Lg, I, D, D, D, I]
    L.or_set_freeze.argtypes = [P, Lg, D]
    L.or_set_advection.argtypes = [P, I]
    L.or_set_incompressible.argtypes = [P, I]
    L.or_set_shear_modulus.argtypes = [P, DP]
    L.or_advect.argtypes = [P, D]
    L.or_apply_increment.argtypes = [P, DP, D, DP]
    L.or_solve_increment.argtypes = [P, C.POINTER(Info)]
    L.or_commit.argtypes = [P]
    L.or_eval.argtypes = [P, DP, DP, DP]
    L.or_field_count.restype = Lg
    L.or_field_count.argtypes = [P, I]
    L.or_get_field.argtypes = [P, I, DP, Lg]
    L.or_set_field.argtypes = [P, I, DP, Lg]
    L.or_pt_params.argtypes = [P, DP, DP, DP]
    L.or_set_start.argtypes = [P, DP]
    L.or_get_eval.argtypes = [P, I, DP, Lg]
    L.or_threads.restype = I
    L.or_threads.argtypes = [I]
    return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def field_shape(ndim, n, name):
    """Natural (C-order, x fastest) shape of a field on the staggered grid."""
    nx, ny = n[0], n[1]
    nz = n[2] if ndim == 3 else 1
    loc = {"vx": (nx + 1, ny, nz), "ux": (nx + 1, ny, nz), "v0x": (nx + 1, ny, nz), "rx": (nx + 1, ny, nz),
           "vy": (nx, ny + 1, nz), "uy": (nx, ny + 1, nz), "v0y": (nx, ny + 1, nz), "ry": (nx, ny + 1, nz),
           "vz": (nx, ny, nz + 1), "uz": (nx, ny, nz + 1), "v0z": (nx, ny, nz + 1), "rz": (nx, ny, nz + 1)}
    if name in loc:
        ex, ey, ez = loc[name]
    elif name in ("txy", "exy"):
        ex, ey, ez = nx + 1, ny + 1, nz
    elif name in ("txz", "exz"):
        ex, ey, ez = nx + 1, ny, nz + 1
    elif name in ("tyz", "eyz"):
        ex, ey, ez = nx, ny + 1, nz + 1
    else:
        ex, ey, ez = nx, ny, nz
    return (ez, ey, ex) if ndim == 3 else (ey, ex)


class Oracle:
    """One staggered grid solved by the FP64 oracle."""

    def __init__(self, ndim, n, L=(1.0, 1.0, 1.0), lib_path=None):
        self.L_ = lib(lib_path)
        self.ndim = ndim
        self.n = tuple(int(x) for x in n[:ndim])
        nn = (C.c_int * 3)(*(list(self.n) + [1] * (3 - ndim)))
        ll = np.ascontiguousarray(list(L[:ndim]) + [1.0] * (3 - ndim), dtype=np.float64)
        self.h = self.L_.or_create(ndim, nn, _dp(ll))
        if not self.h:
            raise ValueError("bad grid")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L_.or_destroy(h)
            self.h = None

    def _chk(self, st, what):
        if st != OK:
            raise RuntimeError("%s failed with status %d" % (what, st))

    def set_material(self, K, G, mu_s, phi_deg, psi_deg, cohesion):
        c = np.ascontiguousarray(cohesion, dtype=np.float64).ravel()
        self._chk(self.L_.or_set_material(self.h, K, G, mu_s, phi_deg, psi_deg, _dp(c)), "set_material")

    def set_solver(self, tol=1e-8, max_iter=1000000, n_chk=100, c_cfl=None, xi=1.0, r_pt=0.5,
                   jaumann=True, advection=False, incompressible=False):
        if c_cfl is None:
            c_cfl = 0.9 / math.sqrt(self.ndim)
        self._chk(self.L_.or_set_solver(self.h, tol, int(max_iter), int(n_chk), c_cfl, xi, r_pt,
                                        int(jaumann)), "set_solver")
        self._chk(self.L_.or_set_advection(self.h, int(bool(advection))), "set_advection")
        self._chk(self.L_.or_set_incompressible(self.h, int(bool(incompressible))), "set_incompressible")

    def set_shear_modulus(self, Gc):
        """Per-cell shear modulus (one value per centre), or None for the
        uniform G of set_material."""
        a = None if Gc is None else np.ascontiguousarray(Gc, dtype=np.float64).ravel()
        if a is not None and a.size != int(np.prod(self.n)):
            raise ValueError("set_shear_modulus: one value per cell centre")
        self._chk(self.L_.or_set_shear_modulus(self.h, _dp(a) if a is not None else None), "set_shear_modulus")

    def advect(self, dt):
        """Advect the old stress (tau_hat, p_hat) over dt with the velocity
        field currently held as the converged velocity (Eq. j1, upwind)."""
        self._chk(self.L_.or_advect(self.h, float(dt)), "advect")

    def set_freeze(self, freeze_iter, freeze_eps=1e-4):
        """Frozen plasticity (Sec. 3.3): freeze the centre return scales at the
        first check with k >= freeze_iter and eps_rel > freeze_eps (0: never)."""
        self._chk(self.L_.or_set_freeze(self.h, int(freeze_iter), float(freeze_eps)), "set_freeze")

    def apply_increment(self, rates, dt, body_force=None):
        r = np.ascontiguousarray(list(rates) + [0.0] * (3 - len(rates)), dtype=np.float64)
        f = None
        if body_force is not None:
            f = np.ascontiguousarray(np.concatenate([np.asarray(b, np.float64).ravel() for b in body_force]))
        self._chk(self.L_.or_apply_increment(self.h, _dp(r), dt, _dp(f) if f is not None else None),
                  "apply_increment")

    def solve_increment(self, commit=True, raise_on_fail=True):
        info = Info()
        st = self.L_.or_solve_increment(self.h, C.byref(info))
        if st != OK and raise_on_fail:
            raise RuntimeError("oracle solve failed: status %d, %s" % (st, info.as_dict()))
        if commit and st == OK:
            self._chk(self.L_.or_commit(self.h), "commit")
        return info.as_dict()

    def eval(self, v_concat):
        v = np.ascontiguousarray(v_concat, dtype=np.float64)
        mr, ms = C.c_double(), C.c_double()
        self._chk(self.L_.or_eval(self.h, _dp(v), C.byref(mr), C.byref(ms)), "eval")
        return mr.value, ms.value

    def eval_stress(self, name):
        """A stress component of the last evaluation ("txx".."tyz", "p"), in
        the field's shape: after eval(v), the physical response of v."""
        comp = {"txx": 0, "tyy": 1, "tzz": 2, "txy": 3, "txz": 4, "tyz": 5, "p": 6}[name]
        shape = field_shape(self.ndim, self.n + (1,), name)
        out = np.empty(int(np.prod(shape)), dtype=np.float64)
        self._chk(self.L_.or_get_eval(self.h, comp, _dp(out), out.size), "get_eval " + name)
        return out.reshape(shape)

    def commit(self):
        self._chk(self.L_.or_commit(self.h), "commit")

    def pt_params(self):
        """(beta_tau, beta_p, velocity step) of the current increment."""
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        self.L_.or_pt_params(self.h, C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    def set_start(self, v_concat):
        """Replace the interior start velocity of the current increment."""
        v = np.ascontiguousarray(v_concat, dtype=np.float64)
        self._chk(self.L_.or_set_start(self.h, _dp(v)), "set_start")

    def get(self, name):
        fid = FIELD_ID[name]
        cnt = self.L_.or_field_count(self.h, fid)
        out = np.empty(max(cnt, 0), dtype=np.float64)
        if cnt > 0:
            self._chk(self.L_.or_get_field(self.h, fid, _dp(out), cnt), "get " + name)
        return out.reshape(field_shape(self.ndim, self.n + (1,), name)) if cnt > 0 else out

    def set(self, name, arr):
        fid = FIELD_ID[name]
        a = np.ascontiguousarray(arr, dtype=np.float64).ravel()
        self._chk(self.L_.or_set_field(self.h, fid, _dp(a), a.size), "set " + name)


def rates_for(load_plane: str, a: float, ndim: int):
    """Diagonal velocity gradient of pure shear in the given plane (Eqs. A7-A9M)."""
    if load_plane == "xy":
        return [a, -a, 0.0][:max(ndim, 2)] if ndim == 2 else [a, -a, 0.0]
    if load_plane == "xz":
        return [a, 0.0, -a]
    raise ValueError(load_plane)


def from_setup(setup, lib_path=None, **solver):
    """An oracle grid initialised from an :class:`ep_inputs.Setup` (on the
    library at lib_path, default the plain build)."""
    o = Oracle(setup.ndim, setup.n, setup.L, lib_path=lib_path)
    o.set_material(setup.K, setup.G, setup.mu_s, setup.phi_deg, setup.psi_deg, setup.cohesion())
    kw = dict(tol=setup.tol)
    kw.update(solver)
    o.set_solver(**kw)
    return o
