"""ctypes binding of ``lib/libep.so`` (the C ABI declared in ``include/ep.h``).

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels.  Importing this module fails loudly when the library has not
been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libep.so")

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_STATE, ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_TIMEOUT = range(8)
STATUS_NAMES = {0: "EP_OK", 1: "EP_ERR_ARG", 2: "EP_ERR_CUDA", 3: "EP_ERR_OOM", 4: "EP_ERR_STATE",
                5: "EP_ERR_NOT_CONVERGED", 6: "EP_ERR_DIVERGED", 7: "EP_ERR_TIMEOUT", 8: "EP_PENDING"}
PENDING = 8


def measure_fp64_peak():
    """FP64 FMA rate of the current device in TFLOP/s (ep_measure_fp64_peak)."""
    t = C.c_double()
    check(None, lib().ep_measure_fp64_peak(C.byref(t)))
    return t.value


def warm_in(ndim):
    """Input channels of the warm-start network (EP_WARM_IN)."""
    return 13 if ndim == 3 else 9


def warm_out(ndim):
    """Output channels of the warm-start network (EP_WARM_OUT)."""
    return 9 if ndim == 3 else 5
FP64, FP32_MIXED = 0, 1
LOAD_XY, LOAD_XZ = 0, 1
KERNEL_AUTO, KERNEL_STAGED, KERNEL_FUSED, KERNEL_FUSED_TMA, KERNEL_FUSED_REG = -1, 0, 1, 2, 3

FIELDS = ["vx", "vy", "vz", "txx", "tyy", "tzz", "txy", "txz", "tyz", "p", "epl",
          "ux", "uy", "uz", "exx", "eyy", "ezz", "exy", "exz", "eyz", "coh", "eii", "scale",
          "v0x", "v0y", "v0z"]
FIELD_ID = {n: i for i, n in enumerate(FIELDS)}


class SolverOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_longlong), ("n_chk", C.c_int),
                ("c_cfl", C.c_double), ("xi", C.c_double), ("r_pt", C.c_double), ("jaumann", C.c_int),
                ("freeze_iter", C.c_longlong), ("freeze_eps", C.c_double), ("advection", C.c_int),
                ("incompressible", C.c_int), ("wait_cycles", C.c_longlong)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_longlong), ("eps_res", C.c_double), ("eps_mom", C.c_double),
                ("eps_tau", C.c_double), ("eps_p", C.c_double), ("eps_rel", C.c_double),
                ("max_r", C.c_double), ("max_sigma", C.c_double), ("n_plastic", C.c_longlong),
                ("sxx_int_centre", C.c_double), ("sxx_int_right", C.c_double), ("ms", C.c_double),
                ("status", C.c_int), ("frozen_at", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class EPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None

# (name, restype, argtypes) of every exported entry point of include/ep.h
_P, _D, _I, _Z = C.c_void_p, C.c_double, C.c_int, C.c_size_t
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)
SIGNATURES = [
    ("ep_workspace_bytes", _I, [_I, _IP, _I, C.POINTER(C.c_size_t)]),
    ("ep_create_grid", _I, [_I, _IP, _DP, _I, _P, _P, _Z, C.POINTER(_P)]),
    ("ep_set_material", _I, [_P, _D, _D, _D, _D, _D, _DP]),
    ("ep_default_solver", _I, [_I, C.POINTER(SolverOpts)]),
    ("ep_set_solver", _I, [_P, C.POINTER(SolverOpts)]),
    ("ep_apply_increment", _I, [_P, _D, _D, _I, _DP, _I]),
    ("ep_apply_increment_rates", _I, [_P, _DP, _D, _DP, _DP]),
    ("ep_solve_increment", _I, [_P, C.POINTER(SolveInfo)]),
    ("ep_solve_chunks", _I, [_P, _I, C.POINTER(SolveInfo)]),
    ("ep_set_shear_modulus", _I, [_P, _DP]),
    ("ep_measure_fp64_peak", _I, [C.POINTER(C.c_double)]),
    ("ep_net_set_output_scale", _I, [_P, _D]),
    ("ep_net_get_output_scale", _I, [_P, C.POINTER(C.c_double)]),
    ("ep_commit_increment", _I, [_P]),
    ("ep_field_count", _I, [_P, _I, C.POINTER(C.c_size_t)]),
    ("ep_get_fields", _I, [_P, _I, _DP, _Z]),
    ("ep_set_fields", _I, [_P, _I, _DP, _Z]),
    ("ep_set_kernel", _I, [_P, _I, _I]),
    ("ep_create_batch", _I, [C.POINTER(_P), _I, C.POINTER(_P)]),
    ("ep_batch_apply_increment", _I, [_P, _DP, _D]),
    ("ep_batch_solve_increment", _I, [_P, C.POINTER(SolveInfo)]),
    ("ep_batch_autotune", _I, [_P, _I, _IP]),
    ("ep_batch_set_tile", _I, [_P, _I]),
    ("ep_batch_time_sweep", _I, [_P, _I, _DP]),
    ("ep_destroy_batch", _I, [_P]),
    ("ep_net_create", _I, [_I, _I, _I, _I, _I, C.c_ulonglong, _P, C.POINTER(_P)]),
    ("ep_net_param_count", _I, [_P, C.POINTER(C.c_longlong)]),
    ("ep_net_get_params", _I, [_P, C.POINTER(C.c_float), C.c_longlong]),
    ("ep_net_set_params", _I, [_P, C.POINTER(C.c_float), C.c_longlong]),
    ("ep_net_forward", _I, [_P, _P, _I, _IP, _P]),
    ("ep_net_forward_static", _I, [_P, _P, _I, _IP, _P]),
    ("ep_net_gradients", _I, [_P, _P, _P, _I, _IP, C.POINTER(C.c_double), C.POINTER(C.c_float), C.c_longlong]),
    ("ep_net_train_step", _I, [_P, _P, _P, _I, _IP, C.c_float, C.POINTER(C.c_double)]),
    ("ep_net_destroy", _I, [_P]),
    ("ep_net_last_error", C.c_char_p, [_P]),
    ("ep_attach_warm_start", _I, [_P, _P, _I]),
    ("ep_warm_dims", _I, [_P, _I, _IP]),
    ("ep_warm_record", _I, [_P, _I]),
    ("ep_warm_features", _I, [_P, _I, _P]),
    ("ep_warm_target", _I, [_P, _I, _P]),
    ("ep_snapshot", _I, [_P]),
    ("ep_restore", _I, [_P]),
    ("ep_time_sweep", _I, [_P, _I, _DP, _I, _IP]),
    ("ep_sweep_bytes_per_cell", _I, [_P, _DP]),
    ("ep_destroy", _I, [_P]),
    ("ep_last_error", C.c_char_p, [_P]),
]


def lib():
    """Load libep.so (raises if it is missing: build it with ``build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libep.so not built at %s; run __graft_entry__.build() or "
                              "paper_2305_01701_gb300.build.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(_DP)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64).ravel()


def check(h, st):
    if st != OK:
        msg = lib().ep_last_error(h)
        raise EPError(st, msg.decode() if msg else "")
    return st


def field_shape(ndim, n, name):
    """Natural C-order shape of a field (x fastest), matching include/ep.h."""
    nx, ny = n[0], n[1]
    nz = n[2] if ndim == 3 else 1
    faces = {"x": (nx + 1, ny, nz), "y": (nx, ny + 1, nz), "z": (nx, ny, nz + 1)}
    if name in ("vx", "ux", "v0x", "vy", "uy", "v0y", "vz", "uz", "v0z"):
        ex, ey, ez = faces[name[-1]]
    elif name in ("txy", "exy"):
        ex, ey, ez = nx + 1, ny + 1, nz
    elif name in ("txz", "exz"):
        ex, ey, ez = nx + 1, ny, nz + 1
    elif name in ("tyz", "eyz"):
        ex, ey, ez = nx, ny + 1, nz + 1
    else:
        ex, ey, ez = nx, ny, nz
    return (ez, ey, ex) if ndim == 3 else (ey, ex)


def workspace_bytes(ndim, n, precision=FP64):
    nn = (C.c_int * 3)(*(list(n[:ndim]) + [1] * (3 - ndim)))
    out = C.c_size_t()
    check(None, lib().ep_workspace_bytes(ndim, nn, precision, C.byref(out)))
    return out.value


class Grid:
    """One staggered grid solved on the GPU through the C ABI.

    ``stream``: an integer cudaStream_t handle (e.g.
    ``torch.cuda.current_stream().cuda_stream``) or None.  ``workspace``: an
    integer device pointer of at least :func:`workspace_bytes` bytes (e.g. the
    data_ptr of a torch uint8 tensor the caller keeps alive) or None.
    """

    def __init__(self, ndim, n, L=(1.0, 1.0, 1.0), precision=FP64, stream=None, workspace=None,
                 workspace_size=0):
        self._L = lib()
        self.ndim = ndim
        self.n = tuple(int(x) for x in n[:ndim])
        self.precision = precision
        nn = (C.c_int * 3)(*(list(self.n) + [1] * (3 - ndim)))
        ll = _f64(list(L[:ndim]) + [1.0] * (3 - ndim))
        h = _P()
        st = self._L.ep_create_grid(ndim, nn, _dp(ll), precision, stream, workspace, workspace_size, C.byref(h))
        check(None, st)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self._L.ep_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_material(self, K, G, mu_s, phi_deg, psi_deg, cohesion):
        c = _f64(cohesion)
        check(self.h, self._L.ep_set_material(self.h, K, G, mu_s, phi_deg, psi_deg, _dp(c)))

    def default_solver(self):
        o = SolverOpts()
        check(self.h, self._L.ep_default_solver(self.ndim, C.byref(o)))
        return o

    def set_shear_modulus(self, G):
        """Per-cell shear modulus (one value per centre), or None for the
        uniform G of set_material."""
        a = None if G is None else _f64(np.asarray(G, dtype=np.float64).ravel())
        if a is not None and a.size != int(np.prod(self.n)):
            raise ValueError("set_shear_modulus: one value per cell centre")
        check(self.h, self._L.ep_set_shear_modulus(self.h, _dp(a)))

    def set_solver(self, tol=1e-8, max_iter=10000000, n_chk=100, c_cfl=None, xi=1.0, r_pt=0.5, jaumann=True,
                   freeze_iter=-1, freeze_eps=1e-4, advection=False, incompressible=False,
                   wait_cycles=0):
        """freeze_iter: frozen plasticity (Sec. 3.3) from this iteration on
        when eps_rel > freeze_eps; -1 the paper's rule (16 n_x above 10^6
        cells), 0 never.  advection: transport the old stress with the last
        converged velocity at the start of each increment (Eq. j1).
        incompressible: Eq. A2ssP2 in place of Eq. A2ssP."""
        o = self.default_solver()
        o.tol = tol
        o.max_iter = int(max_iter)
        o.n_chk = int(n_chk)
        o.c_cfl = c_cfl if c_cfl is not None else 0.9 / math.sqrt(self.ndim)
        o.xi = xi
        o.r_pt = r_pt
        o.jaumann = int(bool(jaumann))
        o.freeze_iter = int(freeze_iter)
        o.freeze_eps = float(freeze_eps)
        o.advection = int(bool(advection))
        o.incompressible = int(bool(incompressible))
        o.wait_cycles = int(wait_cycles)
        check(self.h, self._L.ep_set_solver(self.h, C.byref(o)))

    def apply_increment(self, a, dt, load_plane=LOAD_XY, body_force=None, use_warm_start=False):
        f = None if body_force is None else _f64(np.concatenate([_f64(b) for b in body_force]))
        check(self.h, self._L.ep_apply_increment(self.h, a, dt, load_plane, _dp(f), int(use_warm_start)))

    def apply_increment_rates(self, rates, dt, body_force=None, dv_start=None):
        r = _f64(list(rates) + [0.0] * (3 - len(rates)))
        f = None if body_force is None else _f64(np.concatenate([_f64(b) for b in body_force]))
        dv = None if dv_start is None else _f64(np.concatenate([_f64(b) for b in dv_start]))
        check(self.h, self._L.ep_apply_increment_rates(self.h, _dp(r), dt, _dp(f), _dp(dv)))

    def solve_increment(self, raise_on_fail=True):
        info = SolveInfo()
        st = self._L.ep_solve_increment(self.h, C.byref(info))
        if raise_on_fail:
            check(self.h, st)
        d = info.as_dict()
        d["status"] = st
        return d

    def solve_chunks(self, max_chunks=1, raise_on_fail=True):
        """At most max_chunks chunks of the open increment's iteration; the
        returned dict's "status" is PENDING while the solve is undecided."""
        info = SolveInfo()
        st = self._L.ep_solve_chunks(self.h, int(max_chunks), C.byref(info))
        if raise_on_fail and st != PENDING:
            check(self.h, st)
        d = info.as_dict()
        d["status"] = st
        return d

    def commit_increment(self):
        check(self.h, self._L.ep_commit_increment(self.h))

    def count(self, name):
        c = C.c_size_t()
        check(self.h, self._L.ep_field_count(self.h, FIELD_ID[name], C.byref(c)))
        return c.value

    def get(self, name):
        n = self.count(name)
        out = np.empty(n, dtype=np.float64)
        check(self.h, self._L.ep_get_fields(self.h, FIELD_ID[name], _dp(out), n))
        return out.reshape(field_shape(self.ndim, self.n + (1,), name))

    def set_kernel(self, variant=-1, kz=0):
        """-1 auto, 0 staged (five kernels), 1 fused (cp.async), 2 fused (TMA, 3D),
        3 fused (register z-march, 3D); kz planes per block (0: by grid size)."""
        check(self.h, self._L.ep_set_kernel(self.h, int(variant), int(kz)))

    def snapshot(self):
        check(self.h, self._L.ep_snapshot(self.h))

    def attach_warm_start(self, net, coarsen=1):
        """Use `net` (EP_WARM_IN inputs, EP_WARM_OUT outputs) at coarsening
        `coarsen` for ep_apply_increment(..., use_warm_start=True)."""
        check(self.h, self._L.ep_attach_warm_start(self.h, net.h if net is not None else None, int(coarsen)))

    def warm_dims(self, coarsen=1):
        """Padded coarse grid {X, Y, Z} of the warm-start tensors."""
        dims = (C.c_int * 3)()
        check(self.h, self._L.ep_warm_dims(self.h, int(coarsen), dims))
        return tuple(dims)

    def warm_record(self, on=True):
        """Keep what ep_warm_target needs at every later commit."""
        check(self.h, self._L.ep_warm_record(self.h, int(bool(on))))

    def warm_features(self, out_ptr, coarsen=1):
        """Write the next increment's features to device memory at out_ptr."""
        check(self.h, self._L.ep_warm_features(self.h, int(coarsen), out_ptr))

    def warm_target(self, out_ptr, coarsen=1):
        """Write the last recorded increment's target to device memory at out_ptr."""
        check(self.h, self._L.ep_warm_target(self.h, int(coarsen), out_ptr))

    def restore(self):
        check(self.h, self._L.ep_restore(self.h))

    def set_from(self, name, host_ptr, count):
        """Copy a history field from caller memory at host_ptr (e.g. pinned torch storage)."""
        check(self.h, self._L.ep_set_fields(self.h, FIELD_ID[name], C.cast(host_ptr, _DP), count))

    def get_into(self, name, host_ptr, count):
        """Copy a field into caller memory at host_ptr (e.g. pinned torch storage)."""
        check(self.h, self._L.ep_get_fields(self.h, FIELD_ID[name], C.cast(host_ptr, _DP), count))

    def time_sweep(self, iters=10):
        """Mean ms per launch of each sweep kernel, then of a whole iteration."""
        out = np.zeros(16, dtype=np.float64)
        nk = C.c_int()
        check(self.h, self._L.ep_time_sweep(self.h, int(iters), _dp(out), 16, C.byref(nk)))
        return out[: nk.value + 1].copy()

    def sweep_bytes_per_cell(self):
        b = C.c_double()
        check(self.h, self._L.ep_sweep_bytes_per_cell(self.h, C.byref(b)))
        return b.value

    def set(self, name, arr):
        a = _f64(arr)
        check(self.h, self._L.ep_set_fields(self.h, FIELD_ID[name], _dp(a), a.size))


class Batch:
    """Many 2D grids advanced by one persistent kernel per iteration.

    The grids stay owned by the caller (keep them alive while the batch is
    used); they must be 2D and share precision and n_chk.  Call close()
    before closing the grids: a batch that is garbage-collected without it
    keeps its small device records rather than risk being destroyed after
    its grids.
    """

    def __init__(self, grids):
        self._L = lib()
        self.grids = list(grids)
        arr = (_P * len(self.grids))(*[g.h for g in self.grids])
        b = _P()
        check(None, self._L.ep_create_batch(arr, len(self.grids), C.byref(b)))
        self.h = b

    def close(self):
        if getattr(self, "h", None):
            self._L.ep_destroy_batch(self.h)
            self.h = None

    def apply_increment(self, a, dt):
        rates = _f64(a if np.ndim(a) else [a] * len(self.grids))
        check(None, self._L.ep_batch_apply_increment(self.h, _dp(rates), dt))

    def solve_increment(self, raise_on_fail=True):
        infos = (SolveInfo * len(self.grids))()
        st = self._L.ep_batch_solve_increment(self.h, infos)
        if raise_on_fail:
            check(None, st)
        return [i.as_dict() for i in infos], st

    def autotune(self, iters=20):
        t = C.c_int()
        check(None, self._L.ep_batch_autotune(self.h, int(iters), C.byref(t)))
        return t.value

    def set_tile(self, tile):
        check(None, self._L.ep_batch_set_tile(self.h, int(tile)))

    def time_sweep(self, iters=10):
        """Mean ms of one batched sweep (every grid active) on the open increments."""
        ms = C.c_double()
        check(None, self._L.ep_batch_time_sweep(self.h, int(iters), C.byref(ms)))
        return ms.value


def _ncheck(n, st):
    if st != OK:
        msg = lib().ep_net_last_error(n)
        raise EPError(st, msg.decode() if msg else "")


class Net:
    """The warm-start U-Net (device parameters; tensors are device pointers)."""

    def __init__(self, ndim, in_ch, out_ch, base=32, levels=3, seed=0, stream=None):
        self._L = lib()
        self.ndim, self.in_ch, self.out_ch, self.base, self.levels = ndim, in_ch, out_ch, base, levels
        h = _P()
        _ncheck(None, self._L.ep_net_create(ndim, in_ch, out_ch, base, levels, seed, stream, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self._L.ep_net_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def n_params(self):
        c = C.c_longlong()
        _ncheck(self.h, self._L.ep_net_param_count(self.h, C.byref(c)))
        return c.value

    def get_params(self):
        n = self.n_params()
        out = np.empty(n, dtype=np.float32)
        _ncheck(self.h, self._L.ep_net_get_params(self.h, out.ctypes.data_as(C.POINTER(C.c_float)), n))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _ncheck(self.h, self._L.ep_net_set_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float)), p.size))

    @staticmethod
    def _size(size):
        return (C.c_int * 3)(*(list(size) + [1] * (3 - len(size))))

    def forward(self, x_ptr, N, size, y_ptr):
        _ncheck(self.h, self._L.ep_net_forward(self.h, x_ptr, N, self._size(size), y_ptr))

    def forward_static(self, x_ptr, N, size, y_ptr):
        """forward() with the activations in the library's static device
        array: no allocation, shapes up to the static limit, calls on one
        device must not overlap on the GPU."""
        _ncheck(self.h, self._L.ep_net_forward_static(self.h, x_ptr, N, self._size(size), y_ptr))

    def gradients(self, x_ptr, t_ptr, N, size):
        n = self.n_params()
        g = np.empty(n, dtype=np.float32)
        loss = C.c_double()
        _ncheck(self.h, self._L.ep_net_gradients(self.h, x_ptr, t_ptr, N, self._size(size), C.byref(loss),
                                                  g.ctypes.data_as(C.POINTER(C.c_float)), n))
        return loss.value, g

    def loss(self, x_ptr, t_ptr, N, size):
        """MSE of the network on N samples (ep_net_gradients without the
        gradient copy)."""
        out = C.c_double()
        _ncheck(self.h, self._L.ep_net_gradients(self.h, x_ptr, t_ptr, N, self._size(size), C.byref(out), None, 0))
        return out.value

    def set_output_scale(self, scale):
        _ncheck(self.h, self._L.ep_net_set_output_scale(self.h, float(scale)))

    def output_scale(self):
        out = C.c_double()
        _ncheck(self.h, self._L.ep_net_get_output_scale(self.h, C.byref(out)))
        return out.value

    def train_step(self, x_ptr, t_ptr, N, size, lr):
        loss = C.c_double()
        _ncheck(self.h, self._L.ep_net_train_step(self.h, x_ptr, t_ptr, N, self._size(size), float(lr),
                                                   C.byref(loss)))
        return loss.value
