"""An independent numpy statement of the discrete fixed point that one load
increment of the pseudo-transient iteration converges to, written from the
paper's equations for small grids (test infrastructure; it shares no code with
the oracle or the library).

At pseudo-steady state the pseudo-time derivatives of Eqs. A22P, A2ssP and
A23ssP vanish, so with the relaxation weights (beta_tau, beta_p) of one
implicit pseudo step the iteration stops where the unknowns
    v (interior faces), tau_c (centre deviator), tau_e (interior vertex/edge
    shear deviator), p (centres)
satisfy, for the given history (tau_hat, p_hat) and wall velocities,
    p     = p_hat - K dt div v                                  (Eq. A2ssP)
    T     = beta_tau tau + (1 - beta_tau) tau_tr(v)             (Eq. A23ssP)
    tau_c = s_c T_c,  s_c = min(1, Y / sqrt(J2(T)))             (Sec. 3.3,
            Y = max(0, A p + B c)                                Eqs. A6-A6121lambda)
    tau_e = mean(s of the 4 adjacent centres) T_e
    0     = div(tau - p I)  at interior faces                   (Eq. A22S)
where tau_tr is the Maxwell trial 2 eta_ve (eps_dev + tau_J / (2 G dt)) with
the old stress rotated by the spin of v (Eqs. A41, A5, j1-j14, Appendix A),
J2 squares the shear terms and averages them from the 4 surrounding
vertices/edges to the centre, and free-slip walls carry zero shear.

``solve`` finds the root by Newton's method with a finite-difference
Jacobian, an iteration unrelated to the pseudo-transient one.
"""
from __future__ import annotations

import math

import numpy as np


def dp_coefficients(ndim, phi_deg):
    """Drucker-Prager A, B: 2D Eq. A61 (sin, cos), 3D Eq. A611 (inscribed cone)."""
    sp, cp = math.sin(math.radians(phi_deg)), math.cos(math.radians(phi_deg))
    if ndim == 2:
        return sp, cp
    d = math.sqrt(3.0) * (3.0 - sp)
    return 6.0 * sp / d, 6.0 * cp / d


def _av(a, axes):
    """Mean of the two neighbours along each of `axes` (shrinks them by one)."""
    for ax in axes:
        lo = [slice(None)] * a.ndim
        hi = [slice(None)] * a.ndim
        lo[ax] = slice(None, -1)
        hi[ax] = slice(1, None)
        a = 0.5 * (a[tuple(lo)] + a[tuple(hi)])
    return a


def _d(a, ax, h):
    """Forward difference along axis ax divided by h (shrinks it by one)."""
    return np.diff(a, axis=ax) / h


class Problem:
    """One increment on an nx x ny [x nz] grid of box size L.

    hist: dict with 'v0x', 'v0y'[, 'v0z'] (start velocity, walls included),
    'txx', 'tyy'[, 'tzz'], 'txy'[, 'txz', 'tyz'] (old deviator), 'p' (old
    pressure), 'coh'; arrays in numpy order ([k,] j, i)."""

    def __init__(self, ndim, n, L, K, G, mu_s, phi_deg, dt, beta_tau, hist, jaumann=True):
        self.nd = ndim
        self.n = tuple(n[:ndim])
        self.h = [L[d] / n[d] for d in range(ndim)]
        self.K, self.G, self.dt, self.bt = K, G, dt, beta_tau
        self.eta = G * dt if math.isinf(mu_s) else 1.0 / (1.0 / (G * dt) + 1.0 / mu_s)
        self.c2 = self.eta / (G * dt)
        self.A, self.B = dp_coefficients(ndim, phi_deg)
        self.jaumann = jaumann
        self.hist = {k: np.asarray(v, dtype=np.float64) for k, v in hist.items()}
        # the unknowns: interior faces of each velocity component, the centre
        # deviator components, the interior shear points, the pressure
        vn = ["vx", "vy", "vz"][:ndim]
        self.v_int = []
        for d, name in enumerate(vn):
            full = self.hist["v0" + name[1]]
            self.v_int.append(self._interior_face_slice(d, full.shape))
        self.sh_names = ["txy"] if ndim == 2 else ["txy", "txz", "tyz"]
        self.cn_names = ["txx", "tyy"] if ndim == 2 else ["txx", "tyy", "tzz"]
        self.shapes = []
        for d in range(ndim):
            self.shapes.append(("v", d, self.hist["v0" + "xyz"[d]][self.v_int[d]].shape))
        nc = self.hist["p"].shape
        for d in range(ndim):
            self.shapes.append(("tc", d, nc))
        for c, name in enumerate(self.sh_names):
            self.shapes.append(("te", c, self.hist[name][self._interior_shear_slice(c)].shape))
        self.shapes.append(("p", 0, nc))
        self.sizes = [int(np.prod(s[2])) for s in self.shapes]

    # -- layout helpers ---------------------------------------------------
    def _axis(self, d):
        """numpy axis of spatial dimension d (x is the last axis)."""
        return self.nd - 1 - d

    def _interior_face_slice(self, d, shape):
        sl = [slice(None)] * self.nd
        sl[self._axis(d)] = slice(1, -1)
        return tuple(sl)

    def _shear_dims(self, c):
        """spatial dimensions along which shear component c sits on faces."""
        if self.nd == 2:
            return (0, 1)
        return [(0, 1), (0, 2), (1, 2)][c]

    def _interior_shear_slice(self, c):
        sl = [slice(None)] * self.nd
        for d in self._shear_dims(c):
            sl[self._axis(d)] = slice(1, -1)
        return tuple(sl)

    def pack(self, v, tc, te, p):
        parts = [v[d][self.v_int[d]] for d in range(self.nd)]
        parts += [tc[d] for d in range(self.nd)]
        parts += [te[c][self._interior_shear_slice(c)] for c in range(len(self.sh_names))]
        parts += [p]
        return np.concatenate([np.ravel(a) for a in parts])

    def unpack(self, x):
        out, off = [], 0
        for (kind, d, shp), sz in zip(self.shapes, self.sizes):
            out.append(x[off:off + sz].reshape(shp))
            off += sz
        nd, ns = self.nd, len(self.sh_names)
        v = []
        for d in range(nd):
            full = self.hist["v0" + "xyz"[d]].copy()
            full[self.v_int[d]] = out[d]
            v.append(full)
        tc = out[nd:2 * nd]
        te = []
        for c in range(ns):
            full = np.zeros_like(self.hist[self.sh_names[c]])
            full[self._interior_shear_slice(c)] = out[2 * nd + c]
            te.append(full)
        p = out[2 * nd + ns]
        return v, tc, te, p

    # -- the discrete operators -------------------------------------------
    def rates(self, v):
        """centre normal rates, divergence, shear rates and spins (walls 0)."""
        nd = self.nd
        en = [_d(v[d], self._axis(d), self.h[d]) for d in range(nd)]
        div = sum(en)
        es, om = [], []
        for c in range(len(self.sh_names)):
            a_dim, b_dim = self._shear_dims(c)          # e.g. (x, y) for xy
            # d v_a / d x_b and d v_b / d x_a at the interior shear points
            va = v[a_dim]
            vb = v[b_dim]
            ga = _d(va, self._axis(b_dim), self.h[b_dim])
            gb = _d(vb, self._axis(a_dim), self.h[a_dim])
            sla = [slice(None)] * nd
            sla[self._axis(a_dim)] = slice(1, -1)
            slb = [slice(None)] * nd
            slb[self._axis(b_dim)] = slice(1, -1)
            ga, gb = ga[tuple(sla)], gb[tuple(slb)]
            full_e = np.zeros_like(self.hist[self.sh_names[c]])
            full_w = np.zeros_like(full_e)
            full_e[self._interior_shear_slice(c)] = 0.5 * (ga + gb)
            full_w[self._interior_shear_slice(c)] = 0.5 * (ga - gb)
            es.append(full_e)
            om.append(full_w)
        return en, div, es, om

    def _to_centre(self, a, c):
        """mean of shear component c's 4 points around each centre."""
        return _av(a, [self._axis(d) for d in self._shear_dims(c)])

    def _centres_to_shear(self, a, c):
        """mean of the 4 centres around each interior point of component c,
        placed in the component's full array (walls 0)."""
        full = np.zeros_like(self.hist[self.sh_names[c]])
        full[self._interior_shear_slice(c)] = _av(a, [self._axis(d) for d in self._shear_dims(c)])
        return full

    def _shear_to_shear(self, a, c_from, c_to):
        """mean of component c_from's 4 points nearest each interior point of
        component c_to (3D cross terms), in c_to's full array."""
        # c_from lives on faces along dims F, c_to along dims T; along a dim
        # in F but not T average face->centre (shrink), along a dim in T but
        # not F average centre->face (interior points only)
        F, T = set(self._shear_dims(c_from)), set(self._shear_dims(c_to))
        b = a
        for d in F - T:
            b = _av(b, [self._axis(d)])
        for d in T - F:
            b = _av(b, [self._axis(d)])
        # b now lives on the interior points of c_to along T - F and on all
        # points along the shared dims; keep the interior along every dim of T
        sl = [slice(None)] * self.nd
        for d in T & F:
            sl[self._axis(d)] = slice(1, -1)
        full = np.zeros_like(self.hist[self.sh_names[c_to]])
        full[self._interior_shear_slice(c_to)] = b[tuple(sl)]
        return full

    def rotated_history(self, om):
        """old deviator plus dt times its Jaumann rotation with spin om
        (2D: R_xx = -R_yy = 2 t_xy w_xy, R_xy = w_xy (t_yy - t_xx); 3D:
        Appendix A), products averaged to the target location."""
        H = self.hist
        tn = [H[nm] for nm in self.cn_names]
        ts = [H[nm] for nm in self.sh_names]
        if not self.jaumann:
            return [t.copy() for t in tn], [t.copy() for t in ts]
        dt = self.dt
        if self.nd == 2:
            q = self._to_centre(ts[0] * om[0], 0)
            rn = [tn[0] + dt * 2.0 * q, tn[1] - dt * 2.0 * q]
            rs = [ts[0] + dt * om[0] * self._centres_to_shear(tn[1] - tn[0], 0)]
            return rn, rs
        pxy = self._to_centre(ts[0] * om[0], 0)
        pxz = self._to_centre(ts[1] * om[1], 1)
        pyz = self._to_centre(ts[2] * om[2], 2)
        rn = [tn[0] + dt * 2.0 * (pxy + pxz), tn[1] - dt * 2.0 * (pxy - pyz), tn[2] - dt * 2.0 * (pxz + pyz)]
        S = self._shear_to_shear
        # omega_ij sigma_jk terms, i.e. R_ij = w_ik s_jk + w_jk s_ik
        Rxy = om[0] * self._centres_to_shear(tn[1] - tn[0], 0) + S(ts[2], 2, 0) * S(om[1], 1, 0) \
            + S(ts[1], 1, 0) * S(om[2], 2, 0)
        Rxz = om[1] * self._centres_to_shear(tn[2] - tn[0], 1) + S(ts[2], 2, 1) * S(om[0], 0, 1) \
            - S(ts[0], 0, 1) * S(om[2], 2, 1)
        Ryz = om[2] * self._centres_to_shear(tn[2] - tn[1], 2) - S(ts[0], 0, 2) * S(om[1], 1, 2) \
            - S(ts[1], 1, 2) * S(om[0], 0, 2)
        rs = [ts[0] + dt * Rxy, ts[1] + dt * Rxz, ts[2] + dt * Ryz]
        # free-slip walls keep zero shear
        for c in range(3):
            m = np.zeros_like(rs[c])
            m[self._interior_shear_slice(c)] = 1.0
            rs[c] = rs[c] * m
        return rn, rs

    def residual(self, x):
        """The fixed-point equations at unknowns x (all zero at the root)."""
        v, tc, te, p = self.unpack(x)
        en, div, es, om = self.rates(v)
        rn, rs = self.rotated_history(om)
        e2 = 2.0 * self.eta
        tr_n = [e2 * (en[d] - div / 3.0) + self.c2 * rn[d] for d in range(self.nd)]
        tr_s = [e2 * es[c] + self.c2 * rs[c] for c in range(len(self.sh_names))]
        bt = self.bt
        Tn = [bt * tc[d] + (1.0 - bt) * tr_n[d] for d in range(self.nd)]
        Ts = [bt * te[c] + (1.0 - bt) * tr_s[c] for c in range(len(self.sh_names))]
        J2 = 0.5 * sum(t * t for t in Tn) + sum(self._to_centre(Ts[c], c) ** 2 for c in range(len(Ts)))
        Y = np.maximum(0.0, self.A * p + self.B * self.hist["coh"])
        sj = np.sqrt(J2)
        s = np.where(sj > Y, Y / np.where(sj > 0, sj, 1.0), 1.0)
        F_p = p - (self.hist["p"] - self.K * self.dt * div)
        F_tc = [tc[d] - s * Tn[d] for d in range(self.nd)]
        F_te = [(te[c] - self._centres_to_shear(s, c) * Ts[c])[self._interior_shear_slice(c)]
                for c in range(len(Ts))]
        sig = [tc[d] - p for d in range(self.nd)]
        F_v = []
        for d in range(self.nd):
            r = _d(sig[d], self._axis(d), self.h[d])        # interior faces of component d
            for c, nm in enumerate(self.sh_names):
                dims = self._shear_dims(c)
                if d not in dims:
                    continue
                o = dims[1] if dims[0] == d else dims[0]
                g = _d(te[c], self._axis(o), self.h[o])     # shear point -> face along o
                sl = [slice(None)] * self.nd
                sl[self._axis(d)] = slice(1, -1)
                r = r + g[tuple(sl)]
            F_v.append(r)
        # scale the equations to comparable magnitudes
        ssc = max(1e-300, float(np.abs(self.hist["coh"]).max()))
        parts = [f * (min(self.h) / ssc) for f in F_v] + [f / ssc for f in F_tc] + [f / ssc for f in F_te] + \
                [F_p / ssc]
        return np.concatenate([np.ravel(a) for a in parts]), s

    def solve(self, x0, tol=1e-14, max_newton=60, fd_rel=1e-7):
        """Newton's method with a central finite-difference Jacobian."""
        x = np.array(x0, dtype=np.float64)
        scale = np.ones_like(x)
        off = 0
        vmax = max(np.abs(self.hist["v0" + "xyz"[d]]).max() for d in range(self.nd))
        smax = max(1e-12, float(np.abs(self.hist["coh"]).max()))
        for (kind, _, _), sz in zip(self.shapes, self.sizes):
            scale[off:off + sz] = vmax if kind == "v" else smax
            off += sz
        for it in range(max_newton):
            F, _ = self.residual(x)
            if np.abs(F).max() <= tol:
                return x, it
            J = np.empty((F.size, x.size))
            for q in range(x.size):
                h = fd_rel * scale[q]
                xp = x.copy(); xp[q] += h
                xm = x.copy(); xm[q] -= h
                J[:, q] = (self.residual(xp)[0] - self.residual(xm)[0]) / (2 * h)
            dx = np.linalg.solve(J, -F)
            x = x + dx
            if np.abs(dx / scale).max() <= 1e-15:
                return x, it + 1
        F, _ = self.residual(x)
        raise RuntimeError("Newton did not converge: |F| = %g" % np.abs(F).max())
