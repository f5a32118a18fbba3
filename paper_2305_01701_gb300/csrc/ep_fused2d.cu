// ep_fused2d.cu -- one pseudo-transient iteration of many 2D grids in one
// persistent kernel.
//
// Work items are (instance, tile) pairs; a block takes items in a strided
// loop, skips instances that have converged, and for each item runs the whole
// iteration on a TX x TY tile of cells with a 2-cell halo staged in shared
// memory:
//   vertex spin/strain (Eqs. A41, A5) -> relaxed trials at vertices and
//   centres (Eq. A23ssP with the Jaumann term of Appendix A) -> pressure and
//   Drucker-Prager return at centres (Eqs. A2ssP, A61, A6121lambda) ->
//   vertex deviators -> momentum residual and velocity update (Eqs. A22S,
//   A22P).
// Check iterations also reduce the residual norms of each instance into its
// own record (warp shuffles, one atomic per block and item).  Instances can
// differ in size and material: each carries its own geometry, scalars and
// arrays.  A single grid is a batch of one, so a batched instance and its
// solo solve perform identical arithmetic.
#include <math.h>

#include "ep_internal.cuh"

namespace ep {

namespace {

__device__ __forceinline__ double maxn(double a, double b) { return (a > b || a != a) ? a : b; }

__device__ __forceinline__ void block_max2(double v, unsigned long long *slot) {
  __shared__ unsigned long long sm[32];
  unsigned long long x = (unsigned long long)__double_as_longlong(fabs(v));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, x, o);
    x = x > w ? x : w;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sm[wid] = x;
  __syncthreads();
  if (wid == 0) {
    x = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long w = __shfl_xor_sync(0xffffffffu, x, o);
      x = x > w ? x : w;
    }
    if (lane == 0 && x) atomicMax(slot, x);
  }
}

template <typename T, int TX, int TY>
struct Smem2 {
  static constexpr int W = TX + 4, H = TY + 4, WH = W * H;
  T vx[WH], vy[WH], rq[WH], rd[WH];
  T om[WH], es[WH], txy[WH], tc0[WH], tc1[WH];
  T s[WH], sxx[WH], syy[WH], nxy[WH];
};

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) k_fused2d(const Inst2<T> *insts, const int4 *items, int n_items, int b,
                                                    int check) {
  using Sm = Smem2<T, TX, TY>;
  constexpr int W = Sm::W, H = Sm::H, WH = Sm::WH, NT = TX * TY;
  extern __shared__ __align__(16) unsigned char smem2_raw[];
  Sm &S = *reinterpret_cast<Sm *>(smem2_raw);
  const int o = 1 - b;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4 item = items[it];
    const Inst2<T> &I = insts[item.x];
    if (*(volatile const int *)&I.di->done != 0) continue;   // uniform per block
    const bool frozen = I.di->frozen != 0;
    const Geo &g = I.g;
    const Scal *sc = I.sc;
    const int i0 = item.y * TX, j0 = item.z * TY;
    const int nx = g.nx, ny = g.ny;
    const long long px = g.px;
    const T rdx = (T)g.rdx, rdy = (T)g.rdy, two_eta = (T)sc->two_eta;
    const T bt = (T)sc->bt, ob = (T)1 - bt, bp = (T)sc->bp, obp = (T)sc->obp, KDt = (T)sc->KDt;
    const T Acoef = (T)sc->A, vs = (T)sc->vstep, qr = (T)0.25, third = (T)(1.0 / 3.0);
    const T *u0 = I.u[b][0], *u1 = I.u[b][1];

    __syncthreads();  // the previous item's shared data is no longer read
    // ---- 0. neighbour-read inputs ----
    for (int p = threadIdx.x; p < WH; p += NT) {
      const int a = p % W, bb = p / W;
      const int gi = i0 - 2 + a, gj = j0 - 2 + bb;
      const bool ok = gi >= 0 && gi < g.px && gj >= 0 && gj < g.py;
      const long long e = (long long)gj * px + gi;
      S.vx[p] = ok ? u0[e] : (T)0;
      S.vy[p] = ok ? u1[e] : (T)0;
      S.rq[p] = ok ? I.rq[e] : (T)0;
      S.rd[p] = ok ? I.rd[e] : (T)0;
    }
    __syncthreads();
    // ---- 1. vertex shear strain rate and spin ----
    for (int p = threadIdx.x; p < WH; p += NT) {
      const int a = p % W, bb = p / W;
      const int gi = i0 - 2 + a, gj = j0 - 2 + bb;
      T es = 0, om = 0;
      if (a >= 1 && bb >= 1 && gi >= 1 && gi <= nx - 1 && gj >= 1 && gj <= ny - 1) {
        T x = (S.vx[p] - S.vx[p - W]) * rdy;   // dvx/dy
        T y = (S.vy[p] - S.vy[p - 1]) * rdx;   // dvy/dx
        es = (T)0.5 * (x + y);
        om = (T)0.5 * (x - y);
      }
      S.es[p] = es;
      S.om[p] = om;
    }
    __syncthreads();
    // ---- 2. relaxed trials at vertices and centres ----
    for (int p = threadIdx.x; p < WH; p += NT) {
      const int a = p % W, bb = p / W;
      const int gi = i0 - 2 + a, gj = j0 - 2 + bb;
      const long long e = (long long)gj * px + gi;
      T v = 0;
      if (a >= 1 && bb >= 1 && gi >= 1 && gi <= nx - 1 && gj >= 1 && gj <= ny - 1) {
        T dyx = qr * (S.rd[p - W - 1] + S.rd[p - W] + S.rd[p - 1] + S.rd[p]);
        T tr = I.tbs[e] + two_eta * S.es[p] + S.om[p] * dyx;
        v = bt * I.ss[b][e] + ob * tr;
      }
      S.txy[p] = v;
      T c0 = 0, c1 = 0;
      if (a < W - 1 && bb < H - 1 && gi >= 0 && gi < nx && gj >= 0 && gj < ny) {
        T exx = (S.vx[p + 1] - S.vx[p]) * rdx;
        T eyy = (S.vy[p + W] - S.vy[p]) * rdy;
        T d3 = (exx + eyy) * third;
        T q = qr * (S.rq[p] * S.om[p] + S.rq[p + 1] * S.om[p + 1] + S.rq[p + W] * S.om[p + W] +
                    S.rq[p + W + 1] * S.om[p + W + 1]);
        T t0 = I.tbn[0][e] + two_eta * (exx - d3) + (T)2 * q;
        T t1 = I.tbn[1][e] + two_eta * (eyy - d3) - (T)2 * q;
        c0 = bt * I.sn[b][0][e] + ob * t0;
        c1 = bt * I.sn[b][1][e] + ob * t1;
      }
      S.tc0[p] = c0;
      S.tc1[p] = c1;
    }
    __syncthreads();
    // ---- 3. pressure and return at centres ----
    double sig = 0.0, dtau = 0.0, dp = 0.0;
    for (int p = threadIdx.x; p < WH; p += NT) {
      const int a = p % W, bb = p / W;
      const int gi = i0 - 2 + a, gj = j0 - 2 + bb;
      T s = 0, sx = 0, sy = 0;
      if (a >= 1 && a < W - 1 && bb >= 1 && bb < H - 1 && gi >= 0 && gi < nx && gj >= 0 && gj < ny) {
        const long long e = (long long)gj * px + gi;
        T div = (S.vx[p + 1] - S.vx[p]) * rdx + (S.vy[p + W] - S.vy[p]) * rdy;
        T pr = bp * I.sp[b][e] + obp * (I.pb[e] - KDt * div);
        T txy = qr * (S.txy[p] + S.txy[p + 1] + S.txy[p + W] + S.txy[p + W + 1]);
        T T0 = S.tc0[p], T1 = S.tc1[p];
        T J2 = txy * txy + (T)0.5 * T0 * T0 + (T)0.5 * T1 * T1;
        if (frozen) {
          s = I.s[e];   // frozen plasticity: the held scale (Sec. 3.3)
        } else {
          T sj = sqrt(J2);
          T Y = Acoef * pr + I.yc[e];
          Y = Y > (T)0 ? Y : (T)0;
          s = sj > Y ? Y / sj : (T)1;
        }
        T n0 = s * T0, n1 = s * T1;
        sx = n0 - pr;
        sy = n1 - pr;
        if (a >= 2 && a < W - 2 && bb >= 2 && bb < H - 2) {   // own cell
          I.sn[o][0][e] = n0;
          I.sn[o][1][e] = n1;
          I.sp[o][e] = pr;
          if (!frozen) I.s[e] = s;
          if (check) {
            sig = maxn(sig, maxn(fabs((double)sx), fabs((double)sy)));
            dtau = maxn(dtau, maxn(fabs((double)n0 - (double)I.cn[0][e]), fabs((double)n1 - (double)I.cn[1][e])));
            dp = maxn(dp, fabs((double)pr - (double)I.cp[e]));
            I.cn[0][e] = n0;
            I.cn[1][e] = n1;
            I.cp[e] = pr;
          }
        }
      }
      S.s[p] = s;
      S.sxx[p] = sx;
      S.syy[p] = sy;
    }
    __syncthreads();
    // ---- 4. vertex deviators ----
    for (int p = threadIdx.x; p < WH; p += NT) {
      const int a = p % W, bb = p / W;
      const int gi = i0 - 2 + a, gj = j0 - 2 + bb;
      T v = 0;
      if (a >= 2 && a < W - 1 && bb >= 2 && bb < H - 1 && gi >= 1 && gi <= nx - 1 && gj >= 1 && gj <= ny - 1)
        v = qr * (S.s[p - W - 1] + S.s[p - W] + S.s[p - 1] + S.s[p]) * S.txy[p];
      S.nxy[p] = v;
      if (a >= 2 && a < W - 2 && bb >= 2 && bb < H - 2 && gi < g.px && gj < g.py) {   // own vertex
        const long long e = (long long)gj * px + gi;
        I.ss[o][e] = v;
        if (check) {
          sig = maxn(sig, fabs((double)v));
          dtau = maxn(dtau, fabs((double)v - (double)I.cs[e]));
          I.cs[e] = v;
        }
      }
    }
    __syncthreads();
    // ---- 5. residual and velocity update of the tile's own faces ----
    double rmax = 0.0, du = 0.0, vm = 0.0;
    for (int p = threadIdx.x; p < TX * TY; p += NT) {
      const int a = 2 + p % TX, bb = 2 + p / TX, pp = bb * W + a;
      const int gi = i0 + p % TX, gj = j0 + p / TX;
      if (gi >= g.px || gj >= g.py) continue;
      const long long e = (long long)gj * px + gi;
      // x-face
      T u = S.vx[pp], un = u;
      const bool xin = gi <= nx && gj < ny;
      if (gi >= 1 && gi <= nx - 1 && gj < ny) {
        T R = (S.sxx[pp] - S.sxx[pp - 1]) * rdx + (S.nxy[pp + W] - S.nxy[pp]) * rdy;
        un = u + vs * R;
        if (check) rmax = maxn(rmax, fabs((double)R));
      }
      I.u[o][0][e] = un;
      if (check && xin) {
        du = maxn(du, fabs((double)un - (double)I.uchk[0][e]));
        vm = maxn(vm, fabs(I.v0[0][e] + (double)u));
        I.uchk[0][e] = un;
      }
      // y-face
      u = S.vy[pp];
      un = u;
      const bool yin = gi < nx && gj <= ny;
      if (gj >= 1 && gj <= ny - 1 && gi < nx) {
        T R = (S.syy[pp] - S.syy[pp - W]) * rdy + (S.nxy[pp + 1] - S.nxy[pp]) * rdx;
        un = u + vs * R;
        if (check) rmax = maxn(rmax, fabs((double)R));
      }
      I.u[o][1][e] = un;
      if (check && yin) {
        du = maxn(du, fabs((double)un - (double)I.uchk[1][e]));
        vm = maxn(vm, fabs(I.v0[1][e] + (double)u));
        I.uchk[1][e] = un;
      }
    }
    if (check) {
      block_max2(sig, &I.di->red[RED_SIG]);
      block_max2(dtau, &I.di->red[RED_DTAU]);
      block_max2(dp, &I.di->red[RED_DP]);
      block_max2(rmax, &I.di->red[RED_R]);
      block_max2(du, &I.di->red[RED_DU]);
      block_max2(vm, &I.di->red[RED_V]);
    }
  }
}

}  // namespace

template <typename T, int TX, int TY>
void launch_fused2d_t(const Inst2<T> *insts, const int4 *items, int n_items, int b, int check, int blocks,
                      cudaStream_t st) {
  k_fused2d<T, TX, TY><<<blocks, TX * TY, sizeof(Smem2<T, TX, TY>), st>>>(insts, items, n_items, b, check);
}

template <typename T>
void launch_fused2d(int tile, const Inst2<T> *insts, const int4 *items, int n_items, int b, int check, int blocks,
                    cudaStream_t st) {
  switch (tile) {
    case 0: launch_fused2d_t<T, 32, 8>(insts, items, n_items, b, check, blocks, st); break;
    case 1: launch_fused2d_t<T, 32, 16>(insts, items, n_items, b, check, blocks, st); break;
    case 2: launch_fused2d_t<T, 64, 8>(insts, items, n_items, b, check, blocks, st); break;
    case 3: launch_fused2d_strip<T>(64, insts, items, n_items, b, check, blocks, st); break;
    default: launch_fused2d_strip<T>(32, insts, items, n_items, b, check, blocks, st); break;
  }
}

void fused2d_tile(int tile, int *tx, int *ty) {
  if (tile >= 3) {   // warp strips: 28 written columns, 64 or 32 rows
    *tx = 28;
    *ty = tile == 3 ? 64 : 32;
    return;
  }
  *tx = tile == 2 ? 64 : 32;
  *ty = tile == 1 ? 16 : 8;
}

namespace {
template <typename T>
__global__ void k_check_batch(const Inst2<T> *insts, int n) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) check_one(insts[q].di, insts[q].sc);
}
}  // namespace

template <typename T>
__global__ void k_init_batch(const Inst2<T> *insts, int n, long long max_iter) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  DevInfo *di = insts[q].di;
  for (int r = 0; r < RED_COUNT; ++r) di->red[r] = 0ull;
  di->done = 0;
  di->frozen = 0;
  di->frozen_at = -1;
  di->k_check = 0;
  di->max_iter = max_iter;
  di->iters = 0;
}

template <typename T>
void launch_init_batch(const Inst2<T> *insts, int n, long long max_iter, cudaStream_t st) {
  k_init_batch<T><<<(n + 127) / 128, 128, 0, st>>>(insts, n, max_iter);
}
template void launch_init_batch<float>(const Inst2<float> *, int, long long, cudaStream_t);
template void launch_init_batch<double>(const Inst2<double> *, int, long long, cudaStream_t);

template <typename T>
void launch_check_batch(const Inst2<T> *insts, int n, cudaStream_t st) {
  k_check_batch<T><<<(n + 127) / 128, 128, 0, st>>>(insts, n);
}

template <typename T>
int fused2d_blocks_per_sm(int tile) {
  if (tile >= 3) return fused2d_strip_blocks_per_sm<T>(tile == 3 ? 64 : 32);
  int nb = 0;
  cudaError_t e;
  if (tile == 0)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fused2d<T, 32, 8>, 256, sizeof(Smem2<T, 32, 8>));
  else if (tile == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fused2d<T, 32, 16>, 512, sizeof(Smem2<T, 32, 16>));
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fused2d<T, 64, 8>, 512, sizeof(Smem2<T, 64, 8>));
  return e == cudaSuccess && nb > 0 ? nb : 1;
}

cudaError_t fused2d_configure() {
  cudaError_t e = cudaSuccess;
#define EP_CFG(T, X, Y)                                                                                  \
  if (e == cudaSuccess)                                                                                  \
    e = cudaFuncSetAttribute(k_fused2d<T, X, Y>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                             (int)sizeof(Smem2<T, X, Y>));
  EP_CFG(float, 32, 8) EP_CFG(float, 32, 16) EP_CFG(float, 64, 8)
  EP_CFG(double, 32, 8) EP_CFG(double, 32, 16) EP_CFG(double, 64, 8)
#undef EP_CFG
  return e;
}

template void launch_check_batch<float>(const Inst2<float> *, int, cudaStream_t);
template void launch_check_batch<double>(const Inst2<double> *, int, cudaStream_t);
template int fused2d_blocks_per_sm<float>(int);
template int fused2d_blocks_per_sm<double>(int);
template void launch_fused2d<float>(int, const Inst2<float> *, const int4 *, int, int, int, int, cudaStream_t);
template void launch_fused2d<double>(int, const Inst2<double> *, const int4 *, int, int, int, int, cudaStream_t);

}  // namespace ep
