// ep_fused2d_strip.cu -- the batched 2D iteration with one warp per strip.
//
// Same arithmetic as ep_fused2d.cu (vertex spin and strain rate, relaxed
// trials at vertices and centres with the Jaumann term, pressure and
// Drucker-Prager return at centres, vertex deviators, momentum residual and
// velocity update; Eqs. A41, A5, A23ssP, A2ssP, A61, A6121lambda, A22S,
// A22P), mapped without shared memory or block barriers:
//   * a work item is (instance, strip of 28 columns, segment of `seg` rows);
//     lane a owns column x = i0 - 2 + a (lanes 2..29 are written);
//   * the warp marches the rows y = j0 - 2 .. j1 + 1 of its segment: at row
//     t it forms the vertex quantities of row t, the centres of row t - 1,
//     the vertex deviators of row t - 1 and the velocities of row t - 2;
//   * x +- 1 neighbours are warp shuffles, y - 1 neighbours are registers
//     carried from the previous row; inputs are loaded two rows ahead;
//   * check iterations reduce the residual norms per warp (one atomic per
//     warp, item and norm).
// Warps take items independently, so a block never waits for another warp.
#include <math.h>

#include "ep_internal.cuh"

namespace ep {

namespace {

constexpr int SW = 32;          // columns a warp covers
constexpr int SO = SW - 4;      // columns it writes
constexpr int SWARPS = 8;       // warps per block
constexpr unsigned FULL = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T xm(T v) { return __shfl_up_sync(FULL, v, 1); }
template <typename T>
__device__ __forceinline__ T xp(T v) { return __shfl_down_sync(FULL, v, 1); }

__device__ __forceinline__ double maxn(double a, double b) { return (a > b || a != a) ? a : b; }

// warp-wide max of |v| (NaN kept: its bit pattern is above +inf), one atomic
__device__ __forceinline__ void warp_max(double v, unsigned long long *slot) {
  unsigned long long x = (unsigned long long)__double_as_longlong(fabs(v));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(FULL, x, o);
    x = x > w ? x : w;
  }
  if ((threadIdx.x & 31) == 0 && x) atomicMax(slot, x);
}

template <typename T>
__global__ void __launch_bounds__(SW *SWARPS) k_fused2d_strip(const Inst2<T> *insts, const int4 *items, int n_items,
                                                              int b, int check, int seg) {
  const int a = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  const int o = 1 - b;
  for (int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < n_items; it += warps) {
    const int4 item = items[it];
    const Inst2<T> &I = insts[item.x];
    if (*(volatile const int *)&I.di->done != 0) continue;   // uniform per warp
    const bool frozen = I.di->frozen != 0;
    const Geo &g = I.g;
    const Scal *sc = I.sc;
    const int nx = g.nx, ny = g.ny, py = g.py;
    const long long px = g.px;
    const int i0 = item.y * SO, j0 = item.z * seg, j1 = min(j0 + seg, py);
    const int gi = i0 - 2 + a;
    const bool xin = gi >= 0 && gi < g.px;
    const bool out_col = a >= 2 && a < SW - 2 && xin;
    const T rdx = (T)g.rdx, rdy = (T)g.rdy, two_eta = (T)sc->two_eta;
    const T bt = (T)sc->bt, ob = (T)1 - bt, bp = (T)sc->bp, obp = (T)sc->obp, KDt = (T)sc->KDt;
    const T Acoef = (T)sc->A, vs = (T)sc->vstep, qr = (T)0.25, third = (T)(1.0 / 3.0), hf = (T)0.5;
    const T *u0 = I.u[b][0], *u1 = I.u[b][1];

    auto at = [&](int row) { return (long long)row * px + gi; };
    // FP32 loads read the nearest in-box column and row without a test: a
    // value outside the box only ever enters guarded expressions
    const long long gic = min(max(gi, 0), g.px - 1);
    auto ld = [&](const T *p, int row) -> T {
      if constexpr (sizeof(T) == 4) return p[(long long)min(max(row, 0), py - 1) * px + gic];
      else return (xin && row >= 0 && row < py) ? p[at(row)] : (T)0;
    };

    // inputs two rows ahead (vertex / face arrays of row r, centre arrays of
    // row r - 1): `next` holds row t + 1, `after` row t + 2
    struct Row {
      T vx, vy, rq, rd, tbs, ss, tbn0, tbn1, sn0, sn1, sp, pb, yc;
    };
    auto load_row = [&](int r, Row &w) {
      w.vx = ld(u0, r); w.vy = ld(u1, r); w.rq = ld(I.rq, r); w.rd = ld(I.rd, r);
      w.tbs = ld(I.tbs, r); w.ss = ld(I.ss[b], r);
      const int c = r - 1;
      w.tbn0 = ld(I.tbn[0], c); w.tbn1 = ld(I.tbn[1], c); w.sn0 = ld(I.sn[b][0], c); w.sn1 = ld(I.sn[b][1], c);
      w.sp = ld(I.sp[b], c); w.pb = ld(I.pb, c); w.yc = ld(I.yc, c);
    };
    Row next, after;

    // row history (suffix _1: row t - 1, _2: row t - 2, _3: row t - 3)
    T vx = 0, vy = 0, vx_1 = 0, vy_1 = 0, vx_2 = 0, vy_2 = 0, rd = 0, rd_1 = 0;
    T P_1 = 0, ts_1 = 0, s_2 = 0, sxx_2 = 0, syy_2 = 0, syy_3 = 0, nxy_2 = 0;
    double sig = 0.0, dtau = 0.0, dp = 0.0, rmax = 0.0, du = 0.0, vm = 0.0;

    load_row(j0 - 2, next);
    load_row(j0 - 1, after);
    for (int t = j0 - 2; t < j1 + 2; ++t) {
      const int c = t - 1, u = t - 2;
      vx_2 = vx_1; vy_2 = vy_1; vx_1 = vx; vy_1 = vy; rd_1 = rd;
      vx = next.vx; vy = next.vy; rd = next.rd;
      const T rq = next.rq, tbs = next.tbs, ssv = next.ss;
      const T tbn0 = next.tbn0, tbn1 = next.tbn1, sn0 = next.sn0, sn1 = next.sn1, sp = next.sp, pb = next.pb,
              yc = next.yc;
      next = after;
      if (t + 2 < j1 + 2) load_row(t + 2, after);

      // ---- vertex (gi, t): shear strain rate, spin, relaxed trial ----
      const T vy_xm = xm(vy), rd_xm = xm(rd), rd_1_xm = xm(rd_1);
      T es = 0, om = 0, ts = 0;
      if (a >= 1 && gi >= 1 && gi <= nx - 1 && t >= 1 && t <= ny - 1) {
        const T x = (vx - vx_1) * rdy;   // dvx/dy
        const T y = (vy - vy_xm) * rdx;  // dvy/dx
        es = hf * (x + y);
        om = hf * (x - y);
        const T dyx = qr * (rd_1_xm + rd_1 + rd_xm + rd);
        const T tr = tbs + two_eta * es + om * dyx;
        ts = bt * ssv + ob * tr;
      }
      const T P = rq * om;

      // ---- centre (gi, t - 1): relaxed trial, pressure, return ----
      const T vx_1_xp = xp(vx_1), P_1_xp = xp(P_1), P_xp = xp(P);
      const T ts_xp = xp(ts), ts_1_xp = xp(ts_1);
      T s_1 = 0, sxx_1 = 0, syy_1 = 0;
      if (a < SW - 1 && gi >= 0 && gi < nx && c >= 0 && c < ny) {
        const T exx = (vx_1_xp - vx_1) * rdx;
        const T eyy = (vy - vy_1) * rdy;
        const T d3 = (exx + eyy) * third;
        const T q = qr * (P_1 + P_1_xp + P + P_xp);
        const T t0 = tbn0 + two_eta * (exx - d3) + (T)2 * q;
        const T t1 = tbn1 + two_eta * (eyy - d3) - (T)2 * q;
        const T c0 = bt * sn0 + ob * t0;
        const T c1 = bt * sn1 + ob * t1;
        if (a >= 1) {
          const long long e = at(c);
          const T div = exx + eyy;
          const T pr = bp * sp + obp * (pb - KDt * div);
          const T txy = qr * (ts_1 + ts_1_xp + ts + ts_xp);
          const T J2 = txy * txy + hf * c0 * c0 + hf * c1 * c1;
          if (frozen) {
            s_1 = I.s[e];   // frozen plasticity: the held scale (Sec. 3.3)
          } else {
            T Y = Acoef * pr + yc;
            Y = Y > (T)0 ? Y : (T)0;
            if constexpr (sizeof(T) == 4) {
              // FP32: compare squares, scale with the reciprocal square root
              s_1 = J2 > Y * Y ? Y * rsqrtf(J2) : (T)1;
            } else {
              const T sj = sqrt(J2);
              s_1 = sj > Y ? Y / sj : (T)1;
            }
          }
          const T n0 = s_1 * c0, n1 = s_1 * c1;
          sxx_1 = n0 - pr;
          syy_1 = n1 - pr;
          if (out_col && c >= j0 && c < j1) {   // own cell
            I.sn[o][0][e] = n0;
            I.sn[o][1][e] = n1;
            I.sp[o][e] = pr;
            if (!frozen) I.s[e] = s_1;
            if (check) {
              sig = maxn(sig, maxn(fabs((double)sxx_1), fabs((double)syy_1)));
              dtau = maxn(dtau, maxn(fabs((double)n0 - (double)I.cn[0][e]), fabs((double)n1 - (double)I.cn[1][e])));
              dp = maxn(dp, fabs((double)pr - (double)I.cp[e]));
              I.cn[0][e] = n0;
              I.cn[1][e] = n1;
              I.cp[e] = pr;
            }
          }
        }
      }

      // ---- vertex (gi, t - 1): deviator from the mean of its centre scales ----
      const T s_1_xm = xm(s_1), s_2_xm = xm(s_2);
      T nxy_1 = 0;
      if (a >= 2 && a < SW - 1 && gi >= 1 && gi <= nx - 1 && c >= 1 && c <= ny - 1)
        nxy_1 = qr * (s_2_xm + s_2 + s_1_xm + s_1) * ts_1;
      if (out_col && c >= j0 && c < j1) {   // own vertex (rows below py)
        const long long e = at(c);
        I.ss[o][e] = nxy_1;
        if (check) {
          sig = maxn(sig, fabs((double)nxy_1));
          dtau = maxn(dtau, fabs((double)nxy_1 - (double)I.cs[e]));
          I.cs[e] = nxy_1;
        }
      }

      // ---- faces (gi, t - 2): residual and velocity update ----
      const T sxx_2_xm = xm(sxx_2), nxy_2_xp = xp(nxy_2);
      if (out_col && u >= j0 && u < j1) {
        const long long e = at(u);
        T un = vx_2;
        if (gi >= 1 && gi <= nx - 1 && u < ny) {
          const T R = (sxx_2 - sxx_2_xm) * rdx + (nxy_1 - nxy_2) * rdy;
          un = vx_2 + vs * R;
          if (check) rmax = maxn(rmax, fabs((double)R));
        }
        I.u[o][0][e] = un;
        if (check && gi <= nx && u < ny) {
          du = maxn(du, fabs((double)un - (double)I.uchk[0][e]));
          vm = maxn(vm, fabs(I.v0[0][e] + (double)vx_2));
          I.uchk[0][e] = un;
        }
        un = vy_2;
        if (u >= 1 && u <= ny - 1 && gi < nx) {
          const T R = (syy_2 - syy_3) * rdy + (nxy_2_xp - nxy_2) * rdx;
          un = vy_2 + vs * R;
          if (check) rmax = maxn(rmax, fabs((double)R));
        }
        I.u[o][1][e] = un;
        if (check && gi < nx && u <= ny) {
          du = maxn(du, fabs((double)un - (double)I.uchk[1][e]));
          vm = maxn(vm, fabs(I.v0[1][e] + (double)vy_2));
          I.uchk[1][e] = un;
        }
      }

      // ---- carry this row's values one row down ----
      P_1 = P; ts_1 = ts; s_2 = s_1; sxx_2 = sxx_1;
      syy_3 = syy_2; syy_2 = syy_1; nxy_2 = nxy_1;
    }
    if (check) {
      warp_max(sig, &I.di->red[RED_SIG]);
      warp_max(dtau, &I.di->red[RED_DTAU]);
      warp_max(dp, &I.di->red[RED_DP]);
      warp_max(rmax, &I.di->red[RED_R]);
      warp_max(du, &I.di->red[RED_DU]);
      warp_max(vm, &I.di->red[RED_V]);
    }
  }
}

}  // namespace

template <typename T>
void launch_fused2d_strip(int seg, const Inst2<T> *insts, const int4 *items, int n_items, int b, int check,
                          int blocks, cudaStream_t st) {
  k_fused2d_strip<T><<<blocks, SW * SWARPS, 0, st>>>(insts, items, n_items, b, check, seg);
}

template <typename T>
int fused2d_strip_blocks_per_sm(int seg) {
  (void)seg;
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fused2d_strip<T>, SW * SWARPS, 0);
  return e == cudaSuccess && nb > 0 ? nb : 1;
}

template void launch_fused2d_strip<float>(int, const Inst2<float> *, const int4 *, int, int, int, int, cudaStream_t);
template void launch_fused2d_strip<double>(int, const Inst2<double> *, const int4 *, int, int, int, int,
                                           cudaStream_t);
template int fused2d_strip_blocks_per_sm<float>(int);
template int fused2d_strip_blocks_per_sm<double>(int);

}  // namespace ep
