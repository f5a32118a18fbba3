// ep_stages.cu -- the pseudo-transient sweep as five stage kernels.
//
// One pseudo-time iteration (Sec. 3.2) is:
//   strain   : shear strain rate and spin of u on vertices/edges (Eqs. A41, A5)
//   trial    : relaxed trial deviator T = bt tau_k + (1 - bt) tau_tr(u) at
//              centres and edges, tau_tr with the Jaumann-rotated old stress
//              (Eqs. A23ssP, j14, Appendix A)
//   centres  : pressure p = bp p_k + (1 - bp)(pb - K dt div u) (Eq. A2ssP),
//              Drucker-Prager return at centres (Eqs. A61, A6121lambda)
//              (check iterations also measure the stress change since the
//              previous check, for the pseudo-time residuals)
//   edges    : edge deviator = mean of the adjacent centre scales x T
//   velocity : momentum residual (Eq. A22S) and u += R / rho~ (Eq. A22P);
//              check iterations measure the change of u since the previous
//              check (the interval-averaged momentum residual)
// Every quantity is computed exactly once per iteration (no halo
// recomputation), which is what an FP64-bound sweep on GB300 wants.  The
// same kernels with beta = 0 evaluate the physical response for the FP64
// start-of-increment and commit passes.
#include <math.h>

#include "ep_internal.cuh"

namespace ep {

namespace {

constexpr int kThreads = 256;

// max that keeps a NaN from either side (fmax would drop it)
__device__ __forceinline__ double maxn(double a, double b) { return (a > b || a != a) ? a : b; }
// the same in the sweep's type: check-iteration maxima are formed in T and
// widened once per thread (FP64 arithmetic is scarce on this part; the
// difference of two nearby FP32 values is exact in FP32)
template <typename T>
__device__ __forceinline__ T maxt(T a, T b) { return (a > b || a != a) ? a : b; }

__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(fabs(v));
}

// block-wide max of non-negative-double bit patterns, one atomic per block
__device__ __forceinline__ void block_max(unsigned long long v, unsigned long long *slot) {
  __shared__ unsigned long long sm[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = v > w ? v : w;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sm[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
      v = v > w ? v : w;
    }
    if (lane == 0 && v) atomicMax(slot, v);
  }
}

struct Pos {
  int i, j, k;
  long long e;
  bool in;
};

__device__ __forceinline__ Pos position(const Geo &g) {
  Pos p;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  p.in = t < g.box;
  p.e = t;
  p.i = (int)(t % g.px);
  long long r = t / g.px;
  p.j = (int)(r % g.py);
  p.k = (int)(r / g.py);
  return p;
}

__device__ __forceinline__ bool skip(const DevInfo *di) { return di != nullptr && *(volatile const int *)&di->done != 0; }

// ---------------------------------------------------------------------------
template <typename T, int ND>
__global__ void __launch_bounds__(kThreads) k_strain(Geo g, Stage<T> S, const Scal *sc, DevInfo *di) {
  if (skip(di)) return;
  const Pos q = position(g);
  if (!q.in) return;
  const int i = q.i, j = q.j, k = q.k, nx = g.nx, ny = g.ny, nz = g.nz;
  const long long e = q.e, px = g.px, pl = g.plane;
  const T rdx = (T)g.rdx, rdy = (T)g.rdy, rdz = (T)g.rdz, h = (T)0.5;
  if (i > nx || j > ny || k > (ND == 3 ? nz : 0)) return;
  // xy: 2D vertices or 3D xy-edges (k < nz)
  {
    T es = 0, om = 0;
    if ((ND == 2 || k < nz) && i > 0 && i < nx && j > 0 && j < ny) {
      T a = (S.u[0][e] - S.u[0][e - px]) * rdy;   // dvx/dy
      T b = (S.u[1][e] - S.u[1][e - 1]) * rdx;    // dvy/dx
      es = h * (a + b);
      om = h * (a - b);
    }
    S.es[0][e] = es;
    S.om[0][e] = om;
  }
  if (ND == 3) {
    T es = 0, om = 0;  // xz-edges (j < ny)
    if (j < ny && i > 0 && i < nx && k > 0 && k < nz) {
      T a = (S.u[0][e] - S.u[0][e - pl]) * rdz;   // dvx/dz
      T b = (S.u[2][e] - S.u[2][e - 1]) * rdx;    // dvz/dx
      es = h * (a + b);
      om = h * (a - b);
    }
    S.es[1][e] = es;
    S.om[1][e] = om;
    es = 0; om = 0;    // yz-edges (i < nx)
    if (i < nx && j > 0 && j < ny && k > 0 && k < nz) {
      T a = (S.u[1][e] - S.u[1][e - pl]) * rdz;   // dvy/dz
      T b = (S.u[2][e] - S.u[2][e - px]) * rdy;   // dvz/dy
      es = h * (a + b);
      om = h * (a - b);
    }
    S.es[2][e] = es;
    S.om[2][e] = om;
  }
}

// ---------------------------------------------------------------------------
template <typename T, int ND>
__global__ void __launch_bounds__(kThreads) k_trial(Geo g, Stage<T> S, const Scal *sc, DevInfo *di) {
  if (skip(di)) return;
  const Pos q = position(g);
  if (!q.in) return;
  const int i = q.i, j = q.j, k = q.k, nx = g.nx, ny = g.ny, nz = g.nz;
  const long long e = q.e, px = g.px, pl = g.plane;
  if (i > nx || j > ny || k > (ND == 3 ? nz : 0)) return;
  const T rdx = (T)g.rdx, rdy = (T)g.rdy, rdz = (T)g.rdz;
  const T two_eta = (T)sc->two_eta, tbs0 = (T)S.tb_scale, qr = (T)0.25, third = (T)(1.0 / 3.0);
  // per point: 2 eta_ve, the weight c2 of the rotation terms (folded into
  // the rotation weights when the modulus is uniform) and of the base trial
  auto te = [&](int w, long long x) { return S.ge[w] ? S.ge[w][x] : two_eta; };
  auto cr = [&](int w, long long x) { return S.gc[w] ? S.gc[w][x] : (T)1; };
  auto tb = [&](int w, long long x) { return S.tb_c2 && S.gc[w] ? S.gc[w][x] : tbs0; };
  const T bt = S.relax ? (T)sc->bt : (T)0, ob = (T)1 - bt;
  // ---- centre ----
  if (i < nx && j < ny && (ND == 2 || k < nz)) {
    const long long c = e;
    T tr[3];
    if (ND == 2) {
      T exx = (S.u[0][c + 1] - S.u[0][c]) * rdx;
      T eyy = (S.u[1][c + px] - S.u[1][c]) * rdy;
      T d3 = (exx + eyy) * third;
      T qv = qr * (S.rq[0][c] * S.om[0][c] + S.rq[0][c + 1] * S.om[0][c + 1] +
                   S.rq[0][c + px] * S.om[0][c + px] + S.rq[0][c + px + 1] * S.om[0][c + px + 1]);
      const T tw = te(0, c), cc = cr(0, c), tbs = tb(0, c);
      qv = cc * qv;
      tr[0] = tbs * S.tbn[0][c] + tw * (exx - d3) + (T)2 * qv;
      tr[1] = tbs * S.tbn[1][c] + tw * (eyy - d3) - (T)2 * qv;
    } else {
      T exx = (S.u[0][c + 1] - S.u[0][c]) * rdx;
      T eyy = (S.u[1][c + px] - S.u[1][c]) * rdy;
      T ezz = (S.u[2][c + pl] - S.u[2][c]) * rdz;
      T d3 = (exx + eyy + ezz) * third;
      T pxy = qr * (S.rq[0][c] * S.om[0][c] + S.rq[0][c + 1] * S.om[0][c + 1] +
                    S.rq[0][c + px] * S.om[0][c + px] + S.rq[0][c + px + 1] * S.om[0][c + px + 1]);
      T pxz = qr * (S.rq[1][c] * S.om[1][c] + S.rq[1][c + 1] * S.om[1][c + 1] +
                    S.rq[1][c + pl] * S.om[1][c + pl] + S.rq[1][c + pl + 1] * S.om[1][c + pl + 1]);
      T pyz = qr * (S.rq[2][c] * S.om[2][c] + S.rq[2][c + px] * S.om[2][c + px] +
                    S.rq[2][c + pl] * S.om[2][c + pl] + S.rq[2][c + pl + px] * S.om[2][c + pl + px]);
      const T tw = te(0, c), cc = cr(0, c), tbs = tb(0, c);
      pxy = cc * pxy; pxz = cc * pxz; pyz = cc * pyz;
      tr[0] = tbs * S.tbn[0][c] + tw * (exx - d3) + (T)2 * (pxy + pxz);
      tr[1] = tbs * S.tbn[1][c] + tw * (eyy - d3) - (T)2 * (pxy - pyz);
      tr[2] = tbs * S.tbn[2][c] + tw * (ezz - d3) - (T)2 * (pxz + pyz);
    }
#pragma unroll
    for (int d = 0; d < ND; ++d) S.Tn[d][c] = S.relax ? bt * S.son[d][c] + ob * tr[d] : tr[d];
  }
  // ---- vertices (2D) / edges (3D) ----
  if (ND == 2) {
    T v = 0;
    if (i > 0 && i < nx && j > 0 && j < ny) {
      T dyx = qr * (S.rd[0][e - px - 1] + S.rd[0][e - px] + S.rd[0][e - 1] + S.rd[0][e]);
      T tr = tb(1, e) * S.tbs[0][e] + te(1, e) * S.es[0][e] + cr(1, e) * (S.om[0][e] * dyx);
      v = S.relax ? bt * S.sos[0][e] + ob * tr : tr;
    }
    S.Ts[0][e] = v;
  } else {
    T v = 0;  // xy-edge
    if (k < nz && i > 0 && i < nx && j > 0 && j < ny) {
      T dyx = qr * (S.rd[0][e - px - 1] + S.rd[0][e - px] + S.rd[0][e - 1] + S.rd[0][e]);
      T Tyz = qr * (S.rq[2][e - 1] + S.rq[2][e] + S.rq[2][e - 1 + pl] + S.rq[2][e + pl]);
      T Wyz = qr * (S.om[2][e - 1] + S.om[2][e] + S.om[2][e - 1 + pl] + S.om[2][e + pl]);
      T Txz = qr * (S.rq[1][e - px] + S.rq[1][e] + S.rq[1][e - px + pl] + S.rq[1][e + pl]);
      T Wxz = qr * (S.om[1][e - px] + S.om[1][e] + S.om[1][e - px + pl] + S.om[1][e + pl]);
      T tr = tb(1, e) * S.tbs[0][e] + te(1, e) * S.es[0][e] + cr(1, e) * (S.om[0][e] * dyx + Tyz * Wxz + Txz * Wyz);
      v = S.relax ? bt * S.sos[0][e] + ob * tr : tr;
    }
    S.Ts[0][e] = v;
    v = 0;    // xz-edge
    if (j < ny && i > 0 && i < nx && k > 0 && k < nz) {
      T dzx = qr * (S.rd[1][e - pl - 1] + S.rd[1][e - pl] + S.rd[1][e - 1] + S.rd[1][e]);
      T Tyz = qr * (S.rq[2][e - 1] + S.rq[2][e] + S.rq[2][e - 1 + px] + S.rq[2][e + px]);
      T Wyz = qr * (S.om[2][e - 1] + S.om[2][e] + S.om[2][e - 1 + px] + S.om[2][e + px]);
      T Txy = qr * (S.rq[0][e - pl] + S.rq[0][e - pl + px] + S.rq[0][e] + S.rq[0][e + px]);
      T Wxy = qr * (S.om[0][e - pl] + S.om[0][e - pl + px] + S.om[0][e] + S.om[0][e + px]);
      T tr = tb(2, e) * S.tbs[1][e] + te(2, e) * S.es[1][e] + cr(2, e) * (S.om[1][e] * dzx + Tyz * Wxy - Txy * Wyz);
      v = S.relax ? bt * S.sos[1][e] + ob * tr : tr;
    }
    S.Ts[1][e] = v;
    v = 0;    // yz-edge
    if (i < nx && j > 0 && j < ny && k > 0 && k < nz) {
      T dzy = qr * ((S.rd[1][e - pl - px] - S.rd[0][e - pl - px]) + (S.rd[1][e - pl] - S.rd[0][e - pl]) +
                    (S.rd[1][e - px] - S.rd[0][e - px]) + (S.rd[1][e] - S.rd[0][e]));
      T Txy = qr * (S.rq[0][e - pl] + S.rq[0][e - pl + 1] + S.rq[0][e] + S.rq[0][e + 1]);
      T Wxy = qr * (S.om[0][e - pl] + S.om[0][e - pl + 1] + S.om[0][e] + S.om[0][e + 1]);
      T Txz = qr * (S.rq[1][e - px] + S.rq[1][e - px + 1] + S.rq[1][e] + S.rq[1][e + 1]);
      T Wxz = qr * (S.om[1][e - px] + S.om[1][e - px + 1] + S.om[1][e] + S.om[1][e + 1]);
      T tr = tb(3, e) * S.tbs[2][e] + te(3, e) * S.es[2][e] + cr(3, e) * (S.om[2][e] * dzy - Txy * Wxz - Txz * Wxy);
      v = S.relax ? bt * S.sos[2][e] + ob * tr : tr;
    }
    S.Ts[2][e] = v;
  }
}

// ---------------------------------------------------------------------------
template <typename T, int ND>
__global__ void __launch_bounds__(kThreads) k_return_centres(Geo g, Stage<T> S, const Scal *sc, DevInfo *di,
                                                              int check) {
  if (skip(di)) return;
  const Pos q = position(g);
  const int i = q.i, j = q.j, k = q.k;
  const long long c = q.e, px = g.px, pl = g.plane;
  const bool act = q.in && i < g.nx && j < g.ny && (ND == 2 || k < g.nz);
  const bool frozen = di != nullptr && di->frozen;
  T sig = 0, dtau = 0, dp = 0;
  if (act) {
    const T qr = (T)0.25;
    T div = (S.u[0][c + 1] - S.u[0][c]) * (T)g.rdx + (S.u[1][c + px] - S.u[1][c]) * (T)g.rdy;
    if (ND == 3) div += (S.u[2][c + pl] - S.u[2][c]) * (T)g.rdz;
    T p;
    if (S.relax) p = (T)sc->bp * S.sop[c] + (T)sc->obp * (S.pb[c] - (T)sc->KDt * div);
    else p = S.pb[c] - (T)sc->KDt_phys * div;
    T txy = qr * (S.Ts[0][c] + S.Ts[0][c + 1] + S.Ts[0][c + px] + S.Ts[0][c + px + 1]);
    T J2 = txy * txy;
    if (ND == 3) {
      T txz = qr * (S.Ts[1][c] + S.Ts[1][c + 1] + S.Ts[1][c + pl] + S.Ts[1][c + pl + 1]);
      T tyz = qr * (S.Ts[2][c] + S.Ts[2][c + px] + S.Ts[2][c + pl] + S.Ts[2][c + pl + px]);
      J2 += txz * txz + tyz * tyz;
    }
    T tn[3];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      tn[d] = S.Tn[d][c];
      J2 += (T)0.5 * tn[d] * tn[d];
    }
    T s;
    if (frozen) {
      s = S.s[c];   // frozen plasticity: the held scale (Sec. 3.3)
    } else {
      T sj = sqrt(J2);
      T Y = (T)sc->A * p + S.yc[c];
      Y = Y > (T)0 ? Y : (T)0;
      s = sj > Y ? Y / sj : (T)1;
      S.s[c] = s;
    }
    S.snp[c] = p;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      T t = s * tn[d];
      S.snn[d][c] = t;
      if (check) {
        sig = maxt(sig, (T)fabs(t - p));
        if (S.relax) {
          dtau = maxt(dtau, (T)fabs(t - S.cn[d][c]));
          S.cn[d][c] = t;
        }
      }
    }
    if (check && S.relax) {
      dp = (T)fabs(p - S.cp[c]);
      S.cp[c] = p;
    }
    if (check && (isnan(s) || isnan(p))) sig = (T)NAN;
  }
  if (check && di) {
    block_max(abs_bits((double)sig), &di->red[RED_SIG]);
    block_max(abs_bits((double)dtau), &di->red[RED_DTAU]);
    block_max(abs_bits((double)dp), &di->red[RED_DP]);
  }
}

// ---------------------------------------------------------------------------
template <typename T, int ND>
__global__ void __launch_bounds__(kThreads) k_return_edges(Geo g, Stage<T> S, const Scal *sc, DevInfo *di,
                                                            int check) {
  if (skip(di)) return;
  const Pos q = position(g);
  const int i = q.i, j = q.j, k = q.k, nx = g.nx, ny = g.ny, nz = g.nz;
  const long long e = q.e, px = g.px, pl = g.plane;
  T sig = 0, dtau = 0;
  const T qr = (T)0.25;
  if (q.in && i <= nx && j <= ny && k <= (ND == 3 ? nz : 0)) {
    if (ND == 2) {
      T v = 0;
      if (i > 0 && i < nx && j > 0 && j < ny)
        v = qr * (S.s[e - px - 1] + S.s[e - px] + S.s[e - 1] + S.s[e]) * S.Ts[0][e];
      S.sns[0][e] = v;
      if (check) {
        sig = (T)fabs(v);
        if (S.relax) {
          dtau = (T)fabs(v - S.cs[0][e]);
          S.cs[0][e] = v;
        }
      }
    } else {
      T v0 = 0, v1 = 0, v2 = 0;
      if (k < nz && i > 0 && i < nx && j > 0 && j < ny)
        v0 = qr * (S.s[e - px - 1] + S.s[e - px] + S.s[e - 1] + S.s[e]) * S.Ts[0][e];
      if (j < ny && i > 0 && i < nx && k > 0 && k < nz)
        v1 = qr * (S.s[e - pl - 1] + S.s[e - pl] + S.s[e - 1] + S.s[e]) * S.Ts[1][e];
      if (i < nx && j > 0 && j < ny && k > 0 && k < nz)
        v2 = qr * (S.s[e - pl - px] + S.s[e - pl] + S.s[e - px] + S.s[e]) * S.Ts[2][e];
      S.sns[0][e] = v0;
      S.sns[1][e] = v1;
      S.sns[2][e] = v2;
      if (check) {
        sig = maxt((T)fabs(v0), maxt((T)fabs(v1), (T)fabs(v2)));
        if (S.relax) {
          dtau = maxt((T)fabs(v0 - S.cs[0][e]), maxt((T)fabs(v1 - S.cs[1][e]), (T)fabs(v2 - S.cs[2][e])));
          S.cs[0][e] = v0;
          S.cs[1][e] = v1;
          S.cs[2][e] = v2;
        }
      }
    }
  }
  if (check && di) {
    block_max(abs_bits((double)sig), &di->red[RED_SIG]);
    block_max(abs_bits((double)dtau), &di->red[RED_DTAU]);
  }
}

// ---------------------------------------------------------------------------
template <typename T, int ND>
__global__ void __launch_bounds__(kThreads) k_velocity(Geo g, Stage<T> S, const Scal *sc, DevInfo *di,
                                                        int check) {
  if (skip(di)) return;
  const Pos q = position(g);
  const int i = q.i, j = q.j, k = q.k, nx = g.nx, ny = g.ny, nz = g.nz;
  const long long e = q.e, px = g.px, pl = g.plane;
  const T rdx = (T)g.rdx, rdy = (T)g.rdy, rdz = (T)g.rdz, vs = (T)sc->vstep;
  T rmax = 0, du = 0;
  double vm = 0.0;   // |v0 + u| needs the FP64 base velocity
  if (q.in && i <= nx && j <= ny && k <= (ND == 3 ? nz : 0)) {
    // x-faces: i <= nx, j < ny, k < nz
    if (j < ny && (ND == 2 || k < nz)) {
      T u = S.u[0][e], un = u;
      if (i > 0 && i < nx) {
        T R = ((S.snn[0][e] - S.snp[e]) - (S.snn[0][e - 1] - S.snp[e - 1])) * rdx +
              (S.sns[0][e + px] - S.sns[0][e]) * rdy;
        if (ND == 3) R += (S.sns[1][e + pl] - S.sns[1][e]) * rdz;
        if (S.f[0]) R += S.f[0][e];
        un = u + vs * R;
        if (check) rmax = (T)fabs(R);
      }
      S.uo[0][e] = un;
      if (check) {
        du = (T)fabs(un - S.uchk[0][e]);
        vm = fabs(S.v0[0][e] + (double)u);
        S.uchk[0][e] = un;
      }
    } else {
      S.uo[0][e] = S.u[0][e];
    }
    // y-faces: i < nx, j <= ny, k < nz
    if (i < nx && (ND == 2 || k < nz)) {
      T u = S.u[1][e], un = u;
      if (j > 0 && j < ny) {
        T R = ((S.snn[1][e] - S.snp[e]) - (S.snn[1][e - px] - S.snp[e - px])) * rdy +
              (S.sns[0][e + 1] - S.sns[0][e]) * rdx;
        if (ND == 3) R += (S.sns[2][e + pl] - S.sns[2][e]) * rdz;
        if (S.f[1]) R += S.f[1][e];
        un = u + vs * R;
        if (check) rmax = maxt(rmax, (T)fabs(R));
      }
      S.uo[1][e] = un;
      if (check) {
        du = maxt(du, (T)fabs(un - S.uchk[1][e]));
        vm = maxn(vm, fabs(S.v0[1][e] + (double)u));
        S.uchk[1][e] = un;
      }
    } else {
      S.uo[1][e] = S.u[1][e];
    }
    if (ND == 3) {
      // z-faces: i < nx, j < ny, k <= nz
      if (i < nx && j < ny) {
        T u = S.u[2][e], un = u;
        if (k > 0 && k < nz) {
          T R = ((S.snn[2][e] - S.snp[e]) - (S.snn[2][e - pl] - S.snp[e - pl])) * rdz +
                (S.sns[1][e + 1] - S.sns[1][e]) * rdx + (S.sns[2][e + px] - S.sns[2][e]) * rdy;
          if (S.f[2]) R += S.f[2][e];
          un = u + vs * R;
          if (check) rmax = maxt(rmax, (T)fabs(R));
        }
        S.uo[2][e] = un;
        if (check) {
          du = maxt(du, (T)fabs(un - S.uchk[2][e]));
          vm = maxn(vm, fabs(S.v0[2][e] + (double)u));
          S.uchk[2][e] = un;
        }
      } else {
        S.uo[2][e] = S.u[2][e];
      }
    }
  }
  if (check && di) {
    block_max(abs_bits((double)rmax), &di->red[RED_R]);
    block_max(abs_bits((double)du), &di->red[RED_DU]);
    block_max(abs_bits(vm), &di->red[RED_V]);
  }
}


// Convergence decision after a check iteration (Sec. 4.2 measures).
__global__ void k_check(DevInfo *di, const Scal *sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  check_one(di, sc);
}

inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

template <typename T>
void launch_strain(const Geo &g, const Stage<T> &S, const Scal *sc, DevInfo *di, cudaStream_t st) {
  if (g.ndim == 2) k_strain<T, 2><<<blocks_for(g.box), kThreads, 0, st>>>(g, S, sc, di);
  else k_strain<T, 3><<<blocks_for(g.box), kThreads, 0, st>>>(g, S, sc, di);
}
template <typename T>
void launch_trial(const Geo &g, const Stage<T> &S, const Scal *sc, DevInfo *di, cudaStream_t st) {
  if (g.ndim == 2) k_trial<T, 2><<<blocks_for(g.box), kThreads, 0, st>>>(g, S, sc, di);
  else k_trial<T, 3><<<blocks_for(g.box), kThreads, 0, st>>>(g, S, sc, di);
}
template <typename T>
void launch_return_centres(const Geo &g, const Stage<T> &S, const Scal *sc, DevInfo *di, int check,
                           cudaStream_t st) {
  if (g.ndim == 2) k_return_centres<T, 2><<<blocks_for(g.box), kThreads, 0, st>>>(g, S, sc, di, check);
  else k_return_centres<T, 3><<<blocks_for(g.box), kThreads, 0, st>>>(g, S, sc, di, check);
}
template <typename T>
void launch_return_edges(const Geo &g, const Stage<T> &S, const Scal *sc, DevInfo *di, int check,
                         cudaStream_t st) {
  if (g.ndim == 2) k_return_edges<T, 2><<<blocks_for(g.box), kThreads, 0, st>>>(g, S, sc, di, check);
  else k_return_edges<T, 3><<<blocks_for(g.box), kThreads, 0, st>>>(g, S, sc, di, check);
}
template <typename T>
void launch_velocity(const Geo &g, const Stage<T> &S, const Scal *sc, DevInfo *di, int check,
                     cudaStream_t st) {
  if (g.ndim == 2) k_velocity<T, 2><<<blocks_for(g.box), kThreads, 0, st>>>(g, S, sc, di, check);
  else k_velocity<T, 3><<<blocks_for(g.box), kThreads, 0, st>>>(g, S, sc, di, check);
}
void launch_check(DevInfo *di, const Scal *sc, cudaStream_t st) { k_check<<<1, 32, 0, st>>>(di, sc); }

#define EP_INST(T)                                                                                      \
  template void launch_strain<T>(const Geo &, const Stage<T> &, const Scal *, DevInfo *, cudaStream_t); \
  template void launch_trial<T>(const Geo &, const Stage<T> &, const Scal *, DevInfo *, cudaStream_t);  \
  template void launch_return_centres<T>(const Geo &, const Stage<T> &, const Scal *, DevInfo *, int,   \
                                         cudaStream_t);                                                 \
  template void launch_return_edges<T>(const Geo &, const Stage<T> &, const Scal *, DevInfo *, int,     \
                                       cudaStream_t);                                                   \
  template void launch_velocity<T>(const Geo &, const Stage<T> &, const Scal *, DevInfo *, int, cudaStream_t);
EP_INST(float)
EP_INST(double)
#undef EP_INST

}  // namespace ep
