// ep_fused3d_tma.cu -- the fused 3D iteration with every plane's inputs
// streamed by the tensor-memory accelerator.
//
// Same arithmetic and z-march as ep_fused3d.cu (spin, relaxed trial, centre
// return, edge return, velocity update; Eqs. A5, A23ssP, A2ssP, A6121lambda,
// A22S, A22P), but all 23 input arrays of a plane (velocity increment,
// rotation weights, old stress state, base trial, pressures, B c) arrive as
// one cp.async.bulk.tensor box each: (TX + 8) x (TY + 4) elements from
// x = i0 - 4 (16-byte aligned) and y = j0 - 2, zero outside the box.  One
// elected thread issues plane t + 1 while the block computes plane t; the
// copies of a plane complete on one of two mbarriers.  Every wait is bounded:
// a timeout marks the grid's record (status 4) and the block returns.
#include <cuda.h>
#include <math.h>

#include "ep_internal.cuh"

namespace ep {

namespace {

constexpr int TX = 32;
constexpr int RU = 4;   // velocity increment: planes t-2 .. t, t+1 in flight
constexpr int RC = 3;   // rotation weights / centre-plane state: t-1, t, t+1
constexpr int RF = 2;   // face-plane state: t, t+1

enum {
  A_VX, A_VY, A_VZ,
  A_RQXY, A_RQXZ, A_RQYZ, A_RD0, A_RD1,
  A_SOXZ, A_SOYZ, A_TBXZ, A_TBYZ,                        // face-plane own arrays
  A_SON0, A_SON1, A_SON2, A_TBN0, A_TBN1, A_TBN2,         // centre-plane own arrays
  A_SOXY, A_TBXY, A_SOP, A_PB, A_YC,
  A_COUNT
};

struct Maps {
  CUtensorMap m[A_COUNT];
};

template <typename T, int TY>
struct Lay {
  static constexpr int BW = TX + 8, BH = TY + 4, BQ = BW * BH;  // TMA tile (elements)
  static constexpr int W = TX + 4, H = TY + 4, WH = W * H;      // computed window
};

template <typename T, int TY>
struct SmemT {
  static constexpr int BQ = Lay<T, TY>::BQ;
  alignas(128) T in_u[3][RU][BQ];
  alignas(128) T in_c[5][RC][BQ];
  alignas(128) T in_f[4][RF][BQ];
  alignas(128) T in_o[11][RC][BQ];
  T oxy[2][BQ], oxz[2][BQ], oyz[2][BQ];
  T exy[2][BQ], exz[BQ], eyz[BQ];
  T txy[BQ], txz[2][BQ], tyz[2][BQ], tc[3][BQ];
  T s[2][BQ];
  T sxx[2][BQ], syy[2][BQ], szz[3][BQ];
  T nxy[2][BQ], nxz[2][BQ], nyz[2][BQ];
  alignas(8) unsigned long long bar[2];
};

__device__ __forceinline__ int rs(int lev, int R) { return ((lev % R) + R) % R; }
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned long long *b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(unsigned long long *b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(unsigned long long *b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: gives up after `limit` SM cycles (by default 2^31, about
// 1 s at 2 GHz, far above any copy's latency)
constexpr long long WAIT_DEFAULT = 1ll << 31;
// test_wait polls without suspending the thread, so that the bound, not
// the hardware's own suspend window, decides when the wait gives up
__device__ __forceinline__ bool bar_test(unsigned long long *b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_wait(unsigned long long *b, unsigned parity, long long limit = WAIT_DEFAULT) {
  const long long t0 = clock64();
  if (limit < WAIT_DEFAULT) {
    while (!bar_test(b, parity))
      if (clock64() - t0 > limit) return false;
    return true;
  }
  while (!bar_try(b, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *map, int x, int y, int z,
                                         unsigned long long *b) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::
          "r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(b))
      : "memory");
}

template <typename T, int TY>
__device__ __forceinline__ void issue_plane(SmemT<T, TY> &S, const Maps &M, int i0, int j0, int lev) {
  unsigned long long *b = &S.bar[lev & 1];
  constexpr unsigned bytes = A_COUNT * Lay<T, TY>::BQ * sizeof(T);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  bar_expect(b, bytes);
  const int x = i0 - 4, y = j0 - 2;
  const int su = rs(lev, RU), sc = rs(lev, RC), sf = rs(lev, RF);
  for (int a = 0; a < 3; ++a) tma_load(S.in_u[a][su], &M.m[A_VX + a], x, y, lev, b);
  for (int a = 0; a < 5; ++a) tma_load(S.in_c[a][sc], &M.m[A_RQXY + a], x, y, lev, b);
  for (int a = 0; a < 4; ++a) tma_load(S.in_f[a][sf], &M.m[A_SOXZ + a], x, y, lev, b);
  for (int a = 0; a < 11; ++a) tma_load(S.in_o[a][sc], &M.m[A_SON0 + a], x, y, lev, b);
}

template <typename T>
struct Out3 {
  T *snn[3], *sns[3], *snp, *uo[3];
  const T *s;   // centre return scales (read when plasticity is frozen)
};

template <typename T, int TY>
__global__ void __launch_bounds__(TX *TY, 1)
    k_fused3d_tma(const __grid_constant__ Maps M, Out3<T> O, Geo g, const Scal *sc, DevInfo *di, int kz) {
  using L = Lay<T, TY>;
  constexpr int BW = L::BW, W = L::W, H = L::H, WH = L::WH, NT = TX * TY;
  if (di != nullptr && *(volatile const int *)&di->done != 0) return;
  const bool frozen = di != nullptr && di->frozen;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SmemT<T, TY> &S = *reinterpret_cast<SmemT<T, TY> *>(smem_raw);
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int kb = blockIdx.z * kz, ke = min(kb + kz, g.pz);
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const T rdx = (T)g.rdx, rdy = (T)g.rdy, rdz = (T)g.rdz;
  const T two_eta = (T)sc->two_eta, bt = (T)sc->bt, ob = (T)1 - bt;
  const T bp = (T)sc->bp, obp = (T)sc->obp, KDt = (T)sc->KDt, Acoef = (T)sc->A;
  const T vs = (T)sc->vstep, qr = (T)0.25, third = (T)(1.0 / 3.0), hf = (T)0.5;
  const long long px = g.px;
  const bool leader = threadIdx.x == 0;

  for (int q = threadIdx.x; q < L::BQ; q += NT) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      S.oxy[r][q] = 0; S.oxz[r][q] = 0; S.oyz[r][q] = 0; S.exy[r][q] = 0;
      S.txz[r][q] = 0; S.tyz[r][q] = 0; S.s[r][q] = 0; S.sxx[r][q] = 0; S.syy[r][q] = 0;
      S.nxy[r][q] = 0; S.nxz[r][q] = 0; S.nyz[r][q] = 0;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) S.szz[r][q] = 0;
  }
  if (leader) {
    bar_init(&S.bar[0]);
    bar_init(&S.bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (leader) issue_plane<T, TY>(S, M, i0, j0, kb - 2);
  unsigned phase[2] = {0u, 0u};

  const long long wait_limit = sc->wait_cycles > 0 ? sc->wait_cycles : WAIT_DEFAULT;
  for (int t = kb - 2; t < ke + 2; ++t) {
    const bool ok = bar_wait(&S.bar[t & 1], phase[t & 1], wait_limit);
    phase[t & 1] ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (leader && di) atomicExch(&di->done, 4);
      // wait once more for this plane's copies (bounded by the default
      // limit whatever the option), so that none is in flight when the
      // block's shared memory is released, then leave
      if (!ok) bar_wait(&S.bar[t & 1], phase[t & 1] ^ 1u);
      return;
    }
    if (leader && t + 1 < ke + 2) issue_plane<T, TY>(S, M, i0, j0, t + 1);

    const int u0 = rs(t, RU), um1 = rs(t - 1, RU), um2 = rs(t - 2, RU);
    const int c0 = rs(t, RC), cm1 = rs(t - 1, RC), f0 = rs(t, RF);
    const int o0 = rs(t, 2), om1 = rs(t - 1, 2);
    const T *vx0 = S.in_u[0][u0], *vy0 = S.in_u[1][u0], *vz0 = S.in_u[2][u0];
    const T *vx1 = S.in_u[0][um1], *vy1 = S.in_u[1][um1], *vz1 = S.in_u[2][um1];
    const T *rqxy0 = S.in_c[0][c0], *rqxz0 = S.in_c[1][c0], *rqyz0 = S.in_c[2][c0], *rd00 = S.in_c[3][c0],
            *rd10 = S.in_c[4][c0];
    const T *rqxy1 = S.in_c[0][cm1], *rqxz1 = S.in_c[1][cm1], *rqyz1 = S.in_c[2][cm1], *rd01 = S.in_c[3][cm1],
            *rd11 = S.in_c[4][cm1];

    // ---- 1. shear strain rate and spin: xy plane t, xz/yz face-plane t ----
    for (int p = threadIdx.x; p < WH; p += NT) {
      const int a = p % W, b = p / W, q = b * BW + a + 2;
      const int gi = i0 - 2 + a, gj = j0 - 2 + b;
      T es = 0, om = 0;
      if (a >= 1 && b >= 1 && t >= 0 && t < nz && gi >= 1 && gi <= nx - 1 && gj >= 1 && gj <= ny - 1) {
        T x = (vx0[q] - vx0[q - BW]) * rdy;
        T y = (vy0[q] - vy0[q - 1]) * rdx;
        es = hf * (x + y); om = hf * (x - y);
      }
      S.exy[o0][q] = es; S.oxy[o0][q] = om;
      es = 0; om = 0;
      if (a >= 1 && t >= 1 && t <= nz - 1 && gi >= 1 && gi <= nx - 1 && gj >= 0 && gj < ny) {
        T x = (vx0[q] - vx1[q]) * rdz;
        T y = (vz0[q] - vz0[q - 1]) * rdx;
        es = hf * (x + y); om = hf * (x - y);
      }
      S.exz[q] = es; S.oxz[o0][q] = om;
      es = 0; om = 0;
      if (b >= 1 && t >= 1 && t <= nz - 1 && gi >= 0 && gi < nx && gj >= 1 && gj <= ny - 1) {
        T x = (vy0[q] - vy1[q]) * rdz;
        T y = (vz0[q] - vz0[q - BW]) * rdy;
        es = hf * (x + y); om = hf * (x - y);
      }
      S.eyz[q] = es; S.oyz[o0][q] = om;
    }
    __syncthreads();

    // ---- 2. relaxed trials: xz/yz face-plane t, xy and centres plane t-1 ----
    const int lc = t - 1;
    const T *soxz = S.in_f[0][f0], *soyz = S.in_f[1][f0], *tbxz = S.in_f[2][f0], *tbyz = S.in_f[3][f0];
    const T *son0 = S.in_o[0][cm1], *son1 = S.in_o[1][cm1], *son2 = S.in_o[2][cm1];
    const T *tbn0 = S.in_o[3][cm1], *tbn1 = S.in_o[4][cm1], *tbn2 = S.in_o[5][cm1];
    const T *soxy = S.in_o[6][cm1], *tbxy = S.in_o[7][cm1];
    for (int p = threadIdx.x; p < WH; p += NT) {
      const int a = p % W, b = p / W, q = b * BW + a + 2;
      const int gi = i0 - 2 + a, gj = j0 - 2 + b;
      T v = 0;
      if (a >= 1 && b < H - 1 && t >= 1 && t <= nz - 1 && gi >= 1 && gi <= nx - 1 && gj >= 0 && gj < ny) {
        T dzx = qr * (rd11[q - 1] + rd11[q] + rd10[q - 1] + rd10[q]);
        T Tyz = qr * (rqyz0[q - 1] + rqyz0[q] + rqyz0[q - 1 + BW] + rqyz0[q + BW]);
        T Wyz = qr * (S.oyz[o0][q - 1] + S.oyz[o0][q] + S.oyz[o0][q - 1 + BW] + S.oyz[o0][q + BW]);
        T Txy = qr * (rqxy1[q] + rqxy1[q + BW] + rqxy0[q] + rqxy0[q + BW]);
        T Wxy = qr * (S.oxy[om1][q] + S.oxy[om1][q + BW] + S.oxy[o0][q] + S.oxy[o0][q + BW]);
        T tr = tbxz[q] + two_eta * S.exz[q] + (S.oxz[o0][q] * dzx + Tyz * Wxy - Txy * Wyz);
        v = bt * soxz[q] + ob * tr;
      }
      S.txz[o0][q] = v;
      v = 0;
      if (a < W - 1 && b >= 1 && t >= 1 && t <= nz - 1 && gi >= 0 && gi < nx && gj >= 1 && gj <= ny - 1) {
        T dzy = qr * ((rd11[q - BW] - rd01[q - BW]) + (rd11[q] - rd01[q]) + (rd10[q - BW] - rd00[q - BW]) +
                      (rd10[q] - rd00[q]));
        T Txy = qr * (rqxy1[q] + rqxy1[q + 1] + rqxy0[q] + rqxy0[q + 1]);
        T Wxy = qr * (S.oxy[om1][q] + S.oxy[om1][q + 1] + S.oxy[o0][q] + S.oxy[o0][q + 1]);
        T Txz = qr * (rqxz0[q - BW] + rqxz0[q - BW + 1] + rqxz0[q] + rqxz0[q + 1]);
        T Wxz = qr * (S.oxz[o0][q - BW] + S.oxz[o0][q - BW + 1] + S.oxz[o0][q] + S.oxz[o0][q + 1]);
        T tr = tbyz[q] + two_eta * S.eyz[q] + (S.oyz[o0][q] * dzy - Txy * Wxz - Txz * Wxy);
        v = bt * soyz[q] + ob * tr;
      }
      S.tyz[o0][q] = v;
      v = 0;
      if (a >= 1 && b >= 1 && lc >= 0 && lc < nz && gi >= 1 && gi <= nx - 1 && gj >= 1 && gj <= ny - 1) {
        T dyx = qr * (rd01[q - BW - 1] + rd01[q - BW] + rd01[q - 1] + rd01[q]);
        T Tyz = qr * (rqyz1[q - 1] + rqyz1[q] + rqyz0[q - 1] + rqyz0[q]);
        T Wyz = qr * (S.oyz[om1][q - 1] + S.oyz[om1][q] + S.oyz[o0][q - 1] + S.oyz[o0][q]);
        T Txz = qr * (rqxz1[q - BW] + rqxz1[q] + rqxz0[q - BW] + rqxz0[q]);
        T Wxz = qr * (S.oxz[om1][q - BW] + S.oxz[om1][q] + S.oxz[o0][q - BW] + S.oxz[o0][q]);
        T tr = tbxy[q] + two_eta * S.exy[om1][q] + (S.oxy[om1][q] * dyx + Tyz * Wxz + Txz * Wyz);
        v = bt * soxy[q] + ob * tr;
      }
      S.txy[q] = v;
      T c0v = 0, c1v = 0, c2v = 0;
      if (a < W - 1 && b < H - 1 && lc >= 0 && lc < nz && gi >= 0 && gi < nx && gj >= 0 && gj < ny) {
        T exx = (vx1[q + 1] - vx1[q]) * rdx;
        T eyy = (vy1[q + BW] - vy1[q]) * rdy;
        T ezz = (vz0[q] - vz1[q]) * rdz;
        T d3 = (exx + eyy + ezz) * third;
        T pxy = qr * (rqxy1[q] * S.oxy[om1][q] + rqxy1[q + 1] * S.oxy[om1][q + 1] +
                      rqxy1[q + BW] * S.oxy[om1][q + BW] + rqxy1[q + BW + 1] * S.oxy[om1][q + BW + 1]);
        T pxz = qr * (rqxz1[q] * S.oxz[om1][q] + rqxz1[q + 1] * S.oxz[om1][q + 1] + rqxz0[q] * S.oxz[o0][q] +
                      rqxz0[q + 1] * S.oxz[o0][q + 1]);
        T pyz = qr * (rqyz1[q] * S.oyz[om1][q] + rqyz1[q + BW] * S.oyz[om1][q + BW] + rqyz0[q] * S.oyz[o0][q] +
                      rqyz0[q + BW] * S.oyz[o0][q + BW]);
        T t0 = tbn0[q] + two_eta * (exx - d3) + (T)2 * (pxy + pxz);
        T t1 = tbn1[q] + two_eta * (eyy - d3) - (T)2 * (pxy - pyz);
        T t2 = tbn2[q] + two_eta * (ezz - d3) - (T)2 * (pxz + pyz);
        c0v = bt * son0[q] + ob * t0;
        c1v = bt * son1[q] + ob * t1;
        c2v = bt * son2[q] + ob * t2;
      }
      S.tc[0][q] = c0v; S.tc[1][q] = c1v; S.tc[2][q] = c2v;
    }
    __syncthreads();

    // ---- 3. pressure and return at centres of plane t-1 ----
    const int s1 = rs(lc, 2), z1 = rs(lc, 3);
    const T *sop = S.in_o[8][cm1], *pbp = S.in_o[9][cm1], *ycp = S.in_o[10][cm1];
    for (int p = threadIdx.x; p < WH; p += NT) {
      const int a = p % W, b = p / W, q = b * BW + a + 2;
      const int gi = i0 - 2 + a, gj = j0 - 2 + b;
      T s = 0, sx = 0, sy = 0, sz = 0;
      if (a >= 1 && a < W - 1 && b >= 1 && b < H - 1 && lc >= 0 && lc < nz && gi >= 0 && gi < nx && gj >= 0 &&
          gj < ny) {
        T div = (vx1[q + 1] - vx1[q]) * rdx + (vy1[q + BW] - vy1[q]) * rdy + (vz0[q] - vz1[q]) * rdz;
        T pr = bp * sop[q] + obp * (pbp[q] - KDt * div);
        T txy = qr * (S.txy[q] + S.txy[q + 1] + S.txy[q + BW] + S.txy[q + BW + 1]);
        T txz = qr * (S.txz[om1][q] + S.txz[om1][q + 1] + S.txz[o0][q] + S.txz[o0][q + 1]);
        T tyz = qr * (S.tyz[om1][q] + S.tyz[om1][q + BW] + S.tyz[o0][q] + S.tyz[o0][q + BW]);
        T T0 = S.tc[0][q], T1 = S.tc[1][q], T2 = S.tc[2][q];
        T J2 = txy * txy + txz * txz + tyz * tyz + hf * T0 * T0 + hf * T1 * T1 + hf * T2 * T2;
        if (frozen) {
          s = O.s[((long long)lc * g.py + gj) * px + gi];
        } else {
          T sj = sqrt(J2);
          T Y = Acoef * pr + ycp[q];
          Y = Y > (T)0 ? Y : (T)0;
          s = sj > Y ? Y / sj : (T)1;
        }
        T n0 = s * T0, n1 = s * T1, n2 = s * T2;
        sx = n0 - pr; sy = n1 - pr; sz = n2 - pr;
        if (a >= 2 && a < W - 2 && b >= 2 && b < H - 2 && lc >= kb && lc < ke) {
          const long long ec = ((long long)lc * g.py + gj) * px + gi;
          O.snn[0][ec] = n0; O.snn[1][ec] = n1; O.snn[2][ec] = n2; O.snp[ec] = pr;
        }
      }
      S.s[s1][q] = s; S.sxx[s1][q] = sx; S.syy[s1][q] = sy; S.szz[z1][q] = sz;
    }
    __syncthreads();

    // ---- 4. new edge deviators: xy plane t-1, xz/yz face-plane t-1 ----
    const int sm2 = rs(lc - 1, 2);
    for (int p = threadIdx.x; p < WH; p += NT) {
      const int a = p % W, b = p / W, q = b * BW + a + 2;
      const int gi = i0 - 2 + a, gj = j0 - 2 + b;
      T vxy = 0, vxz = 0, vyz = 0;
      const bool inner = a >= 2 && a < W - 1 && b >= 2 && b < H - 1;
      if (inner && lc >= 0 && lc < nz && gi >= 1 && gi <= nx - 1 && gj >= 1 && gj <= ny - 1)
        vxy = qr * (S.s[s1][q - BW - 1] + S.s[s1][q - BW] + S.s[s1][q - 1] + S.s[s1][q]) * S.txy[q];
      if (inner && lc >= 1 && lc <= nz - 1 && gi >= 1 && gi <= nx - 1 && gj >= 0 && gj < ny)
        vxz = qr * (S.s[sm2][q - 1] + S.s[sm2][q] + S.s[s1][q - 1] + S.s[s1][q]) * S.txz[om1][q];
      if (inner && lc >= 1 && lc <= nz - 1 && gi >= 0 && gi < nx && gj >= 1 && gj <= ny - 1)
        vyz = qr * (S.s[sm2][q - BW] + S.s[sm2][q] + S.s[s1][q - BW] + S.s[s1][q]) * S.tyz[om1][q];
      S.nxy[s1][q] = vxy; S.nxz[s1][q] = vxz; S.nyz[s1][q] = vyz;
      if (a >= 2 && a < W - 2 && b >= 2 && b < H - 2 && lc >= kb && lc < ke && gi < g.px && gj < g.py) {
        const long long e = ((long long)lc * g.py + gj) * px + gi;
        O.sns[0][e] = vxy; O.sns[1][e] = vxz; O.sns[2][e] = vyz;
      }
    }
    __syncthreads();

    // ---- 5. residual and velocity update of plane t-2 ----
    const int lu = t - 2;
    if (lu >= kb && lu < ke) {
      const int q2 = rs(lu, 2), q1 = rs(lu + 1, 2), z2 = rs(lu, 3), z3 = rs(lu - 1, 3);
      const T *ux = S.in_u[0][um2], *uy = S.in_u[1][um2], *uz = S.in_u[2][um2];
      for (int p = threadIdx.x; p < TX * TY; p += NT) {
        const int q = (2 + p / TX) * BW + 4 + p % TX;
        const int gi = i0 + p % TX, gj = j0 + p / TX;
        if (gi >= g.px || gj >= g.py) continue;
        const long long e = ((long long)lu * g.py + gj) * px + gi;
        T u = ux[q], un = u;
        if (gi >= 1 && gi <= nx - 1 && gj < ny && lu < nz) {
          T R = (S.sxx[q2][q] - S.sxx[q2][q - 1]) * rdx + (S.nxy[q2][q + BW] - S.nxy[q2][q]) * rdy +
                (S.nxz[q1][q] - S.nxz[q2][q]) * rdz;
          un = u + vs * R;
        }
        O.uo[0][e] = un;
        u = uy[q]; un = u;
        if (gj >= 1 && gj <= ny - 1 && gi < nx && lu < nz) {
          T R = (S.syy[q2][q] - S.syy[q2][q - BW]) * rdy + (S.nxy[q2][q + 1] - S.nxy[q2][q]) * rdx +
                (S.nyz[q1][q] - S.nyz[q2][q]) * rdz;
          un = u + vs * R;
        }
        O.uo[1][e] = un;
        u = uz[q]; un = u;
        if (lu >= 1 && lu <= nz - 1 && gi < nx && gj < ny) {
          T R = (S.szz[z2][q] - S.szz[z3][q]) * rdz + (S.nxz[q2][q + 1] - S.nxz[q2][q]) * rdx +
                (S.nyz[q2][q + BW] - S.nyz[q2][q]) * rdy;
          un = u + vs * R;
        }
        O.uo[2][e] = un;
      }
    }
  }
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
  }
  return fn;
}

template <typename T, int TY>
bool encode(CUtensorMap *m, const Geo &g, const void *base) {
  EncodeTiled fn = encoder();
  if (!fn || !base) return false;
  cuuint64_t dims[3] = {(cuuint64_t)g.px, (cuuint64_t)g.py, (cuuint64_t)g.pz};
  cuuint64_t strides[2] = {(cuuint64_t)g.px * sizeof(T), (cuuint64_t)g.plane * sizeof(T)};
  cuuint32_t box[3] = {(cuuint32_t)Lay<T, TY>::BW, (cuuint32_t)Lay<T, TY>::BH, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                  const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <typename T>
constexpr int tma_ty() { return sizeof(T) == 4 ? 8 : 2; }

}  // namespace

// One fused iteration with TMA plane streaming: reads buffer b of the stage,
// writes 1 - b.  The tensor maps are encoded on the host at launch (and
// captured by value in a graph).  Returns false if a map could not be made.
template <typename T>
bool launch_fused3d_tma(const Geo &g, const Stage<T> &S, const Scal *sc, const DevInfo *di, int kz, cudaStream_t st) {
  constexpr int TY = tma_ty<T>();
  Maps M;
  const void *src[A_COUNT] = {S.u[0], S.u[1], S.u[2], S.rq[0], S.rq[1], S.rq[2], S.rd[0], S.rd[1],
                              S.sos[1], S.sos[2], S.tbs[1], S.tbs[2], S.son[0], S.son[1], S.son[2],
                              S.tbn[0], S.tbn[1], S.tbn[2], S.sos[0], S.tbs[0], S.sop, S.pb, S.yc};
  for (int a = 0; a < A_COUNT; ++a)
    if (!encode<T, TY>(&M.m[a], g, src[a])) return false;
  Out3<T> O;
  for (int d = 0; d < 3; ++d) { O.snn[d] = S.snn[d]; O.sns[d] = S.sns[d]; O.uo[d] = S.uo[d]; }
  O.snp = S.snp;
  O.s = S.s;
  kz = fused3d_kz(g, TX, TY, kz);
  dim3 grid((g.px + TX - 1) / TX, (g.py + TY - 1) / TY, (g.pz + kz - 1) / kz);
  k_fused3d_tma<T, TY><<<grid, TX * TY, sizeof(SmemT<T, TY>), st>>>(M, O, g, sc, const_cast<DevInfo *>(di), kz);
  return true;
}

cudaError_t fused3d_tma_configure() {
  if (!encoder()) return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(k_fused3d_tma<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(SmemT<float, 8>));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fused3d_tma<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(SmemT<double, 2>));
}

size_t fused3d_tma_smem_bytes(bool fp64) { return fp64 ? sizeof(SmemT<double, 2>) : sizeof(SmemT<float, 8>); }

template bool launch_fused3d_tma<float>(const Geo &, const Stage<float> &, const Scal *, const DevInfo *, int,
                                        cudaStream_t);
template bool launch_fused3d_tma<double>(const Geo &, const Stage<double> &, const Scal *, const DevInfo *, int,
                                         cudaStream_t);

}  // namespace ep
