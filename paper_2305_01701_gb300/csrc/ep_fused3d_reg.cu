// ep_fused3d_reg.cu -- the fused 3D iteration with the z-march held in
// registers.
//
// Same arithmetic and z-march as ep_fused3d.cu (spin, relaxed trial, centre
// return, edge return, velocity update; Eqs. A5, A23ssP, A2ssP, A6121lambda,
// A22S, A22P), mapped so that almost no neighbour value goes through shared
// memory:
//   * a block covers a window of 32 x H columns (x, y) of the box and walks
//     them through a chunk of z-planes; lane a owns window column x = i0-2+a,
//     warp b owns row y = j0-2+b; the inner 28 x (H-4) columns are written;
//   * x +- 1 neighbours are warp shuffles of registers;
//   * y +- 1 neighbours are rows of shared memory, each written once by its
//     owner (two plane slots where a value is read one plane later);
//   * z - 1 neighbours are registers carried from the previous plane;
//   * inputs arrive through plain coalesced loads issued one plane ahead.
// Plane t of the march computes spins at plane t, edge trials at face t and
// plane t-1, centres t-1, edges t-1 and velocities t-2.  Three block barriers
// separate the steps of a plane: the input rows of plane t+1 are published
// before the third barrier of plane t, once every read of plane t's input
// rows lies behind the second.
// Instruction count (the kernel is issue-bound, not bandwidth-bound):
//   * blocks whose whole window lies inside the domain run a copy of the body
//     in which the domain-boundary tests are compile-time true;
//   * FP32 loads take a clamped in-box address and no test: a value read
//     outside the box only ever enters guarded expressions;
//   * the march is unrolled by two planes, so the shared-memory slot of each
//     copy is a compile-time constant;
//   * offsets within an array are 32-bit when the box has fewer than 2^31
//     points (FP32), so an address is one wide multiply-add;
//   * the warps of the window's first and last rows, whose centres are never
//     read, skip the centre step, and the first row's warp skips the xz-edge
//     and centre trials (rows are warp-uniform).
// Check iterations (FP32, CHK = true) also reduce the stopping measures of
// Eqs. Convergence1-3 over the points each block writes, the same point sets
// and the same snapshot updates as the staged check iteration: max|sigma|,
// max|tau - tau_chk|, max|p - p_chk| at centres and edges, max|R|,
// max|u - u_chk| and max|v0 + u| at faces, and they store the centre scales
// (held when plasticity freezes).  One atomic per block and measure.  The
// snapshot values a thread checks in a plane are copied to shared memory with
// cp.async at the plane's start and read after the second barrier, so that
// their memory latency hides behind the plane's first steps.
#include <math.h>

#include <type_traits>

#include "ep_internal.cuh"

namespace ep {

namespace {

constexpr int WX = 32;       // window columns: one per lane
constexpr int OX = WX - 4;   // written columns per block
constexpr unsigned FULL = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T xm(T v) { return __shfl_up_sync(FULL, v, 1); }    // value of column a - 1
template <typename T>
__device__ __forceinline__ T xp(T v) { return __shfl_down_sync(FULL, v, 1); }  // value of column a + 1

// One plane slot of a row-exchanged value: rows -1 .. H of the window, so
// that row b +- 1 is always in bounds (the two pad rows stay zero).
template <typename T, int H>
struct Rows {
  T r[H + 2][WX];
};

template <typename T, int H>
struct SmemR {
  Rows<T, H> u0, u2, rq2, oyz, tsxy;                    // read within the plane
  Rows<T, H> u1[2], rq0[2], rq1[2], rd0[2], rd1[2];     // read at this plane and the next
  Rows<T, H> oxy[2], oxz[2], pxy[2], pyz[2], tsyz[2];
  Rows<T, H> s[2], syy[2], nxy[2], nyz[2];
};

template <typename T>
struct Args {
  const T *u[3], *rq[3], *rd[2];
  const T *son[3], *sos[3], *sop, *tbn[3], *tbs[3], *pb, *yc;
  T *snn[3], *sns[3], *snp, *uo[3];
  T *s;   // centre return scales (read when plasticity is frozen, written by checks)
  T *cn[3], *cs[3], *cp, *uchk[3];   // state at the previous check (check iterations)
  const double *v0[3];               // start velocity (check iterations)
};

// a check iteration's snapshot values, one slot per thread, after SmemR
template <typename T, int H>
struct ChkSlots {
  T cn[3][WX * H], cs[3][WX * H], cp[WX * H], uchk[3][WX * H];
  double v0[3][WX * H];
};

__device__ __forceinline__ void cp_async_el(float *smem, const float *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_el(double *smem, const double *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

template <typename T>
__device__ __forceinline__ T maxt(T a, T b) { return (a > b || a != a) ? a : b; }
// |x| in the type of x (no round trip through double for FP32)
__device__ __forceinline__ float absv(float x) { return fabsf(x); }
__device__ __forceinline__ double absv(double x) { return fabs(x); }

// block-wide max of a non-negative value as its IEEE bits (integer order; a
// NaN sorts above infinity), one atomic per block
__device__ __forceinline__ void block_max_bits(double v, unsigned long long *slot) {
  __shared__ unsigned long long part[32];
  unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(FULL, b, o);
    b = b > w ? b : w;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) part[wid] = b;
  __syncthreads();
  if (wid == 0) {
    b = lane < (int)(blockDim.x >> 5) ? part[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(FULL, b, o);
      b = b > w ? b : w;
    }
    if (lane == 0 && b) atomicMax(slot, b);
  }
}

// INT: every column of the block's window lies strictly inside the domain
// (1 <= x, y index <= n - 1), so the domain-boundary tests fold away.
// Off: the integer type of offsets within an array.  CHK: a check iteration.
template <typename T, int H, bool INT, typename Off, bool CHK>
__device__ __forceinline__ void reg_body(const Args<T> &A, const Geo &g, const Scal *sc, DevInfo *di, bool frozen,
                                         int kz, unsigned char *smem_raw) {
  SmemR<T, H> &S = *reinterpret_cast<SmemR<T, H> *>(smem_raw);
  ChkSlots<T, H> &C = *reinterpret_cast<ChkSlots<T, H> *>(smem_raw + sizeof(SmemR<T, H>));   // CHK only
  constexpr int W = WX;
  const int a = threadIdx.x & 31, b = threadIdx.x >> 5;
  const int i0 = blockIdx.x * OX, j0 = blockIdx.y * (H - 4);
  const int gi = i0 - 2 + a, gj = j0 - 2 + b;
  const int kb = blockIdx.z * kz, ke = min(kb + kz, g.pz);
  const int nz = g.nz, pz = g.pz;
  const Off px = (Off)g.px, plane = (Off)g.plane;
  const bool inb = INT || (gi >= 0 && gi < g.px && gj >= 0 && gj < g.py);
  const bool gx1 = INT || (gi >= 1 && gi <= g.nx - 1), gy1 = INT || (gj >= 1 && gj <= g.ny - 1);
  const bool gx0 = INT || (gi >= 0 && gi < g.nx), gy0 = INT || (gj >= 0 && gj < g.ny);
  const bool gxl = INT || gi < g.nx, gyl = INT || gj < g.ny;
  // this column's offset in a plane.  FP32 clamps it into the box so that
  // loads need no test (a value outside the box only ever enters guarded
  // expressions); every store and the frozen-scale read are guarded by
  // in-box tests, where the clamped offset is the exact one.  FP64 keeps the
  // tested loads (fewer registers).
  const Off col = sizeof(T) == 4 ? (Off)min(max(gj, 0), g.py - 1) * px + (Off)min(max(gi, 0), g.px - 1)
                                 : (inb ? (Off)gj * px + (Off)gi : (Off)0);

  const bool out_col = a >= 2 && a < W - 2 && b >= 2 && b < H - 2;
  const T rdx = (T)g.rdx, rdy = (T)g.rdy, rdz = (T)g.rdz;
  const T two_eta = (T)sc->two_eta, bt = (T)sc->bt, ob = (T)1 - bt;
  const T bp = (T)sc->bp, obp = (T)sc->obp, KDt = (T)sc->KDt, Acoef = (T)sc->A;
  const T vs = (T)sc->vstep, qr = (T)0.25, third = (T)(1.0 / 3.0), hf = (T)0.5;
  const int rb = b + 1;  // this thread's row in a Rows slot

  // zero the pad rows (never written afterwards)
  {
    T *base = reinterpret_cast<T *>(smem_raw);
    constexpr int n_rows = sizeof(SmemR<T, H>) / sizeof(Rows<T, H>);
    for (int q = threadIdx.x; q < n_rows * 2 * WX; q += WX * H) {
      const int slot = q / (2 * WX), rem = q % (2 * WX);
      const int row = rem < WX ? 0 : H + 1;
      base[(long long)slot * (H + 2) * WX + row * WX + (rem % WX)] = (T)0;
    }
  }

  auto ld = [&](const T *p, int lev) -> T {
    if constexpr (sizeof(T) == 4) return __ldg(p + ((Off)min(max(lev, 0), pz - 1) * plane + col));
    else return (inb && lev >= 0 && lev < pz) ? __ldg(p + ((Off)lev * plane + col)) : (T)0;
  };

  // inputs of the next plane (loaded one plane ahead)
  T n_u0, n_u1, n_u2, n_rq0, n_rq1, n_rq2, n_rd0, n_rd1, n_soxz, n_soyz, n_tbxz, n_tbyz;
  T n_son0, n_son1, n_son2, n_tbn0, n_tbn1, n_tbn2, n_soxy, n_tbxy, n_sop, n_pb, n_yc;
  auto prefetch = [&](int t) {  // face/edge arrays of plane t, centre arrays of plane t - 1
    n_u0 = ld(A.u[0], t); n_u1 = ld(A.u[1], t); n_u2 = ld(A.u[2], t);
    n_rq0 = ld(A.rq[0], t); n_rq1 = ld(A.rq[1], t); n_rq2 = ld(A.rq[2], t);
    n_rd0 = ld(A.rd[0], t); n_rd1 = ld(A.rd[1], t);
    n_soxz = ld(A.sos[1], t); n_soyz = ld(A.sos[2], t); n_tbxz = ld(A.tbs[1], t); n_tbyz = ld(A.tbs[2], t);
    const int c = t - 1;
    n_son0 = ld(A.son[0], c); n_son1 = ld(A.son[1], c); n_son2 = ld(A.son[2], c);
    n_tbn0 = ld(A.tbn[0], c); n_tbn1 = ld(A.tbn[1], c); n_tbn2 = ld(A.tbn[2], c);
    n_soxy = ld(A.sos[0], c); n_tbxy = ld(A.tbs[0], c); n_sop = ld(A.sop, c); n_pb = ld(A.pb, c);
    n_yc = ld(A.yc, c);
  };
  // the row-exchanged inputs of the prefetched plane, into its plane slot
  auto publish = [&](const int slot) {
    S.u0.r[rb][a] = n_u0; S.u2.r[rb][a] = n_u2; S.u1[slot].r[rb][a] = n_u1;
    S.rq0[slot].r[rb][a] = n_rq0; S.rq1[slot].r[rb][a] = n_rq1; S.rq2.r[rb][a] = n_rq2;
    S.rd0[slot].r[rb][a] = n_rd0; S.rd1[slot].r[rb][a] = n_rd1;
  };

  // plane history (suffix: _1 plane t-1, _2 plane t-2, _3 plane t-3)
  T u0 = 0, u1 = 0, u2 = 0, u0_1 = 0, u1_1 = 0, u2_1 = 0, u0_2 = 0, u1_2 = 0, u2_2 = 0;
  T rq0 = 0, rq1 = 0, rq2 = 0, rd0 = 0, rd1 = 0, rq0_1 = 0, rq1_1 = 0, rq2_1 = 0, rd0_1 = 0, rd1_1 = 0;
  T oxy_1 = 0, oxz_1 = 0, oyz_1 = 0, exy_1 = 0, pxy_1 = 0, pxz_1 = 0, pyz_1 = 0;
  T tsxz_1 = 0, tsyz_1 = 0;
  T s_2 = 0;                                   // centre scale, plane t-2
  T sxx_2 = 0, syy_2 = 0, szz_2 = 0, szz_3 = 0;  // centre stress minus pressure
  T nxy_2 = 0, nxz_2 = 0, nyz_2 = 0;           // edge stress, level t-2
  // check iterations: the stopping measures over this block's points
  T c_sig = 0, c_dtau = 0, c_dp = 0, c_r = 0, c_du = 0;
  double c_vm = 0.0;

  prefetch(kb - 2);
  publish(0);
  __syncthreads();
  // the march unrolled by two planes: the slot parity of each copy is a
  // compile-time constant
  auto plane_step = [&](const int t, auto slc) {
    constexpr int sl = decltype(slc)::value, sl1 = sl ^ 1;  // plane slots of t and t - 1
    // ---- 0. take this plane's inputs (their rows are already published) ----
    u0_2 = u0_1; u1_2 = u1_1; u2_2 = u2_1;
    u0_1 = u0; u1_1 = u1; u2_1 = u2;
    u0 = n_u0; u1 = n_u1; u2 = n_u2;
    rq0_1 = rq0; rq1_1 = rq1; rq2_1 = rq2; rd0_1 = rd0; rd1_1 = rd1;
    rq0 = n_rq0; rq1 = n_rq1; rq2 = n_rq2; rd0 = n_rd0; rd1 = n_rd1;
    const T soxz = n_soxz, soyz = n_soyz, tbxz = n_tbxz, tbyz = n_tbyz;
    const T son0 = n_son0, son1 = n_son1, son2 = n_son2, tbn0 = n_tbn0, tbn1 = n_tbn1, tbn2 = n_tbn2;
    const T soxy = n_soxy, tbxy = n_tbxy, sop = n_sop, pb = n_pb, yc = n_yc;
    const bool more = t + 1 < ke + 2;
    if (more) prefetch(t + 1);
    if constexpr (CHK) {   // the snapshot values checked at this plane: levels t-1 (centres, edges), t-2 (faces)
      const int tid = threadIdx.x;
      const Off e1 = (Off)min(max(t - 1, 0), pz - 1) * plane + col, e2 = (Off)min(max(t - 2, 0), pz - 1) * plane + col;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        cp_async_el(&C.cn[d][tid], A.cn[d] + e1);
        cp_async_el(&C.cs[d][tid], A.cs[d] + e1);
        cp_async_el(&C.uchk[d][tid], A.uchk[d] + e2);
        cp_async_el(&C.v0[d][tid], A.v0[d] + e2);
      }
      cp_async_el(&C.cp[tid], A.cp + e1);
      cp_async_commit();
    }

    // ---- 1. shear strain rates and spins at plane t (xy) / face t (xz, yz) ----
    T exy = 0, oxy = 0, exz = 0, oxz = 0, eyz = 0, oyz = 0;
    {
      const T u0_ym = S.u0.r[rb - 1][a], u2_ym = S.u2.r[rb - 1][a];
      const T u1_xm = xm(u1), u2_xm = xm(u2);
      if (a >= 1 && b >= 1 && t >= 0 && t < nz && gx1 && gy1) {
        const T x = (u0 - u0_ym) * rdy, y = (u1 - u1_xm) * rdx;
        exy = hf * (x + y); oxy = hf * (x - y);
      }
      if (a >= 1 && t >= 1 && t <= nz - 1 && gx1 && gy0) {
        const T x = (u0 - u0_1) * rdz, y = (u2 - u2_xm) * rdx;
        exz = hf * (x + y); oxz = hf * (x - y);
      }
      if (b >= 1 && t >= 1 && t <= nz - 1 && gx0 && gy1) {
        const T x = (u1 - u1_1) * rdz, y = (u2 - u2_ym) * rdy;
        eyz = hf * (x + y); oyz = hf * (x - y);
      }
    }
    const T pxy = rq0 * oxy, pxz = rq1 * oxz, pyz = rq2 * oyz;  // rotation products
    S.oxy[sl].r[rb][a] = oxy; S.oxz[sl].r[rb][a] = oxz; S.oyz.r[rb][a] = oyz;
    S.pxy[sl].r[rb][a] = pxy; S.pyz[sl].r[rb][a] = pyz;
    __syncthreads();

    // ---- 2. relaxed trials: faces t (xz, yz), plane t-1 (xy, centres) ----
    const int lc = t - 1;
    T tsxz = 0, tsyz = 0, tsxy = 0, c0v = 0, c1v = 0, c2v = 0, exx = 0, eyy = 0, ezz = 0;
    {
      // shuffles run on every lane, outside the validity branches
      const T rd1_1_xm = xm(rd1_1), rd1_xm = xm(rd1), rd0_1_xm = xm(rd0_1);
      const T rq2_xm = xm(rq2), rq2_1_xm = xm(rq2_1), oyz_xm = xm(oyz), oyz_1_xm = xm(oyz_1);
      const T rq2_yp = S.rq2.r[rb + 1][a], oyz_yp = S.oyz.r[rb + 1][a];
      const T rq2_yp_xm = xm(rq2_yp), oyz_yp_xm = xm(oyz_yp);
      const T rq0_1_yp = S.rq0[sl1].r[rb + 1][a], rq0_yp = S.rq0[sl].r[rb + 1][a];
      const T oxy_1_yp = S.oxy[sl1].r[rb + 1][a], oxy_yp = S.oxy[sl].r[rb + 1][a];
      const T rq0_1_xp = xp(rq0_1), rq0_xp = xp(rq0), oxy_1_xp = xp(oxy_1), oxy_xp = xp(oxy);
      const T rq1_ym = S.rq1[sl].r[rb - 1][a], oxz_ym = S.oxz[sl].r[rb - 1][a];
      const T rq1_xp = xp(rq1), oxz_xp = xp(oxz), rq1_ym_xp = xp(rq1_ym), oxz_ym_xp = xp(oxz_ym);
      const T rd0_1_ym = S.rd0[sl1].r[rb - 1][a], rd1_1_ym = S.rd1[sl1].r[rb - 1][a];
      const T rd0_ym = S.rd0[sl].r[rb - 1][a], rd1_ym = S.rd1[sl].r[rb - 1][a];
      const T rd0_1_ym_xm = xm(rd0_1_ym);
      const T rq1_1_ym = S.rq1[sl1].r[rb - 1][a], oxz_1_ym = S.oxz[sl1].r[rb - 1][a];
      const T u0_1_xp = xp(u0_1), u1_1_yp = S.u1[sl1].r[rb + 1][a];
      const T pxy_1_xp = xp(pxy_1), pxy_1_yp = S.pxy[sl1].r[rb + 1][a];
      const T pxy_1_yp_xp = xp(pxy_1_yp);
      const T pxz_1_xp = xp(pxz_1), pxz_xp = xp(pxz);
      const T pyz_1_yp = S.pyz[sl1].r[rb + 1][a], pyz_yp = S.pyz[sl].r[rb + 1][a];

      if (b >= 1 && b < H - 1 && t >= 1 && t <= nz - 1)
      if (a >= 1 && gx1 && gy0) {
        const T dzx = qr * (rd1_1_xm + rd1_1 + rd1_xm + rd1);
        const T Tyz = qr * (rq2_xm + rq2 + rq2_yp_xm + rq2_yp);
        const T Wyz = qr * (oyz_xm + oyz + oyz_yp_xm + oyz_yp);
        const T Txy = qr * (rq0_1 + rq0_1_yp + rq0 + rq0_yp);
        const T Wxy = qr * (oxy_1 + oxy_1_yp + oxy + oxy_yp);
        const T tr = tbxz + two_eta * exz + (oxz * dzx + Tyz * Wxy - Txy * Wyz);
        tsxz = bt * soxz + ob * tr;
      }
      if (b >= 1 && t >= 1 && t <= nz - 1)
      if (a < W - 1 && gx0 && gy1) {
        const T dzy = qr * ((rd1_1_ym - rd0_1_ym) + (rd1_1 - rd0_1) + (rd1_ym - rd0_ym) + (rd1 - rd0));
        const T Txy = qr * (rq0_1 + rq0_1_xp + rq0 + rq0_xp);
        const T Wxy = qr * (oxy_1 + oxy_1_xp + oxy + oxy_xp);
        const T Txz = qr * (rq1_ym + rq1_ym_xp + rq1 + rq1_xp);
        const T Wxz = qr * (oxz_ym + oxz_ym_xp + oxz + oxz_xp);
        const T tr = tbyz + two_eta * eyz + (oyz * dzy - Txy * Wxz - Txz * Wxy);
        tsyz = bt * soyz + ob * tr;
      }
      if (b >= 1 && lc >= 0 && lc < nz)
      if (a >= 1 && gx1 && gy1) {
        const T dyx = qr * (rd0_1_ym_xm + rd0_1_ym + rd0_1_xm + rd0_1);
        const T Tyz = qr * (rq2_1_xm + rq2_1 + rq2_xm + rq2);
        const T Wyz = qr * (oyz_1_xm + oyz_1 + oyz_xm + oyz);
        const T Txz = qr * (rq1_1_ym + rq1_1 + rq1_ym + rq1);
        const T Wxz = qr * (oxz_1_ym + oxz_1 + oxz_ym + oxz);
        const T tr = tbxy + two_eta * exy_1 + (oxy_1 * dyx + Tyz * Wxz + Txz * Wyz);
        tsxy = bt * soxy + ob * tr;
      }
      if (b >= 1 && b < H - 1 && lc >= 0 && lc < nz)
      if (a < W - 1 && gx0 && gy0) {
        exx = (u0_1_xp - u0_1) * rdx;
        eyy = (u1_1_yp - u1_1) * rdy;
        ezz = (u2 - u2_1) * rdz;
        const T d3 = (exx + eyy + ezz) * third;
        const T Pxy = qr * (pxy_1 + pxy_1_xp + pxy_1_yp + pxy_1_yp_xp);
        const T Pxz = qr * (pxz_1 + pxz_1_xp + pxz + pxz_xp);
        const T Pyz = qr * (pyz_1 + pyz_1_yp + pyz + pyz_yp);
        const T t0 = tbn0 + two_eta * (exx - d3) + (T)2 * (Pxy + Pxz);
        const T t1 = tbn1 + two_eta * (eyy - d3) - (T)2 * (Pxy - Pyz);
        const T t2 = tbn2 + two_eta * (ezz - d3) - (T)2 * (Pxz + Pyz);
        c0v = bt * son0 + ob * t0;
        c1v = bt * son1 + ob * t1;
        c2v = bt * son2 + ob * t2;
      }
    }
    S.tsxy.r[rb][a] = tsxy; S.tsyz[sl].r[rb][a] = tsyz;
    __syncthreads();

    // ---- 3. pressure and return at the centres of plane t-1 ----
    T s_1 = 0, sxx_1 = 0, syy_1 = 0, szz_1 = 0;
    if constexpr (CHK) cp_async_wait_all();   // this thread's own slots
    if (b >= 1 && b < H - 1) {
      const T tsxy_xp = xp(tsxy), tsxy_yp = S.tsxy.r[rb + 1][a];
      const T tsxy_yp_xp = xp(tsxy_yp);
      const T tsxz_1_xp = xp(tsxz_1), tsxz_xp = xp(tsxz);
      const T tsyz_1_yp = S.tsyz[sl1].r[rb + 1][a], tsyz_yp = S.tsyz[sl].r[rb + 1][a];
      if (b >= 1 && b < H - 1 && lc >= 0 && lc < nz)
      if (a >= 1 && a < W - 1 && gx0 && gy0) {
        const T div = exx + eyy + ezz;
        const T pr = bp * sop + obp * (pb - KDt * div);
        const T txy = qr * (tsxy + tsxy_xp + tsxy_yp + tsxy_yp_xp);
        const T txz = qr * (tsxz_1 + tsxz_1_xp + tsxz + tsxz_xp);
        const T tyz = qr * (tsyz_1 + tsyz_1_yp + tsyz + tsyz_yp);
        const T J2 = txy * txy + txz * txz + tyz * tyz + hf * c0v * c0v + hf * c1v * c1v + hf * c2v * c2v;
        if (frozen) {
          s_1 = A.s[(Off)lc * plane + col];
        } else {
          T Y = Acoef * pr + yc;
          Y = Y > (T)0 ? Y : (T)0;
          if (sizeof(T) == 4) {
            // FP32: compare squares and scale with the reciprocal square root
            // only where the return acts (most cells stay elastic)
            s_1 = J2 > Y * Y ? (T)(Y * rsqrtf((float)J2)) : (T)1;
          } else {
            const T sj = sqrt(J2);
            s_1 = sj > Y ? Y / sj : (T)1;
          }
        }
        const T n0 = s_1 * c0v, n1 = s_1 * c1v, n2 = s_1 * c2v;
        sxx_1 = n0 - pr; syy_1 = n1 - pr; szz_1 = n2 - pr;
        if (out_col && lc >= kb && lc < ke) {
          const Off ec = (Off)lc * plane + col;
          A.snn[0][ec] = n0; A.snn[1][ec] = n1; A.snn[2][ec] = n2; A.snp[ec] = pr;
          if constexpr (CHK) {   // a centre of the box (lc < nz, gi < nx, gj < ny hold here)
            if (!frozen) A.s[ec] = s_1;
            c_sig = maxt(c_sig, maxt(absv(n0 - pr), maxt(absv(n1 - pr), absv(n2 - pr))));
            const int tid = threadIdx.x;
            c_dtau = maxt(c_dtau, maxt(absv(n0 - C.cn[0][tid]),
                                       maxt(absv(n1 - C.cn[1][tid]), absv(n2 - C.cn[2][tid]))));
            c_dp = maxt(c_dp, absv(pr - C.cp[tid]));
            A.cn[0][ec] = n0; A.cn[1][ec] = n1; A.cn[2][ec] = n2; A.cp[ec] = pr;
            if (isnan(s_1) || isnan(pr)) c_sig = (T)NAN;
          }
        }
      }
    }
    S.s[sl1].r[rb][a] = s_1; S.syy[sl1].r[rb][a] = syy_1;
    // every read of plane t's input rows lies behind the second barrier
    if (more) publish(sl1);
    __syncthreads();

    // ---- 4. new edge deviators at level t-1 ----
    T nxy_1 = 0, nxz_1 = 0, nyz_1 = 0;
    {
      const T s_1_xm = xm(s_1), s_2_xm = xm(s_2);
      const T s_1_ym = S.s[sl1].r[rb - 1][a], s_2_ym = S.s[sl].r[rb - 1][a];
      const T s_1_ym_xm = xm(s_1_ym);
      const bool inner = a >= 2 && a < W - 1 && b >= 2 && b < H - 1;
      if (inner && lc >= 0 && lc < nz && gx1 && gy1)
        nxy_1 = qr * (s_1_ym_xm + s_1_ym + s_1_xm + s_1) * tsxy;
      if (inner && lc >= 1 && lc <= nz - 1 && gx1 && gy0)
        nxz_1 = qr * (s_2_xm + s_2 + s_1_xm + s_1) * tsxz_1;
      if (inner && lc >= 1 && lc <= nz - 1 && gx0 && gy1)
        nyz_1 = qr * (s_2_ym + s_2 + s_1_ym + s_1) * tsyz_1;
      if (out_col && lc >= kb && lc < ke && inb) {
        const Off e = (Off)lc * plane + col;
        A.sns[0][e] = nxy_1; A.sns[1][e] = nxz_1; A.sns[2][e] = nyz_1;
        if constexpr (CHK) {
          if (gi <= g.nx && gj <= g.ny && lc <= nz) {   // the staged check's edge points
            c_sig = maxt(c_sig, maxt(absv(nxy_1), maxt(absv(nxz_1), absv(nyz_1))));
            const int tid = threadIdx.x;
            c_dtau = maxt(c_dtau, maxt(absv(nxy_1 - C.cs[0][tid]),
                                       maxt(absv(nxz_1 - C.cs[1][tid]), absv(nyz_1 - C.cs[2][tid]))));
            A.cs[0][e] = nxy_1; A.cs[1][e] = nxz_1; A.cs[2][e] = nyz_1;
          }
        }
      }
    }
    S.nxy[sl1].r[rb][a] = nxy_1; S.nyz[sl1].r[rb][a] = nyz_1;

    // ---- 5. residual and velocity update of plane t-2 ----
    {
      const int lu = t - 2;
      const T sxx_2_xm = xm(sxx_2), nxy_2_xp = xp(nxy_2), nxz_2_xp = xp(nxz_2);
      if (out_col && inb && lu >= kb && lu < ke) {
        const T nxy_2_yp = S.nxy[sl].r[rb + 1][a], syy_2_ym = S.syy[sl].r[rb - 1][a];
        const T nyz_2_yp = S.nyz[sl].r[rb + 1][a];
        const Off e = (Off)lu * plane + col;
        T un = u0_2;
        if (gx1 && gyl && lu < nz) {
          const T R = (sxx_2 - sxx_2_xm) * rdx + (nxy_2_yp - nxy_2) * rdy + (nxz_1 - nxz_2) * rdz;
          un = u0_2 + vs * R;
          if constexpr (CHK) c_r = maxt(c_r, absv(R));
        }
        A.uo[0][e] = un;
        if constexpr (CHK) {
          if (gi <= g.nx && gj < g.ny && lu < nz) {   // x-faces
            c_du = maxt(c_du, absv(un - C.uchk[0][threadIdx.x]));
            c_vm = fmax(c_vm, fabs(C.v0[0][threadIdx.x] + (double)u0_2));   // a NaN in u also reaches c_du
            A.uchk[0][e] = un;
          }
        }
        un = u1_2;
        if (gy1 && gxl && lu < nz) {
          const T R = (syy_2 - syy_2_ym) * rdy + (nxy_2_xp - nxy_2) * rdx + (nyz_1 - nyz_2) * rdz;
          un = u1_2 + vs * R;
          if constexpr (CHK) c_r = maxt(c_r, absv(R));
        }
        A.uo[1][e] = un;
        if constexpr (CHK) {
          if (gi < g.nx && gj <= g.ny && lu < nz) {   // y-faces
            c_du = maxt(c_du, absv(un - C.uchk[1][threadIdx.x]));
            c_vm = fmax(c_vm, fabs(C.v0[1][threadIdx.x] + (double)u1_2));
            A.uchk[1][e] = un;
          }
        }
        un = u2_2;
        if (lu >= 1 && lu <= nz - 1 && gxl && gyl) {
          const T R = (szz_2 - szz_3) * rdz + (nxz_2_xp - nxz_2) * rdx + (nyz_2_yp - nyz_2) * rdy;
          un = u2_2 + vs * R;
          if constexpr (CHK) c_r = maxt(c_r, absv(R));
        }
        A.uo[2][e] = un;
        if constexpr (CHK) {
          if (gi < g.nx && gj < g.ny && lu <= nz) {   // z-faces
            c_du = maxt(c_du, absv(un - C.uchk[2][threadIdx.x]));
            c_vm = fmax(c_vm, fabs(C.v0[2][threadIdx.x] + (double)u2_2));
            A.uchk[2][e] = un;
          }
        }
      }
    }

    // ---- carry this plane's values one plane down ----
    oxy_1 = oxy; oxz_1 = oxz; oyz_1 = oyz; exy_1 = exy;
    pxy_1 = pxy; pxz_1 = pxz; pyz_1 = pyz;
    tsxz_1 = tsxz; tsyz_1 = tsyz;
    s_2 = s_1;
    sxx_2 = sxx_1; syy_2 = syy_1; szz_3 = szz_2; szz_2 = szz_1;
    nxy_2 = nxy_1; nxz_2 = nxz_1; nyz_2 = nyz_1;
  };
  int t = kb - 2;
  for (; t + 1 < ke + 2; t += 2) {
    plane_step(t, std::integral_constant<int, 0>{});
    plane_step(t + 1, std::integral_constant<int, 1>{});
  }
  if (t < ke + 2) plane_step(t, std::integral_constant<int, 0>{});
  if constexpr (CHK) {
    block_max_bits((double)c_sig, &di->red[RED_SIG]);
    block_max_bits((double)c_dtau, &di->red[RED_DTAU]);
    block_max_bits((double)c_dp, &di->red[RED_DP]);
    block_max_bits((double)c_r, &di->red[RED_R]);
    block_max_bits((double)c_du, &di->red[RED_DU]);
    block_max_bits(c_vm, &di->red[RED_V]);
  }
}

template <typename T, int H, typename Off, bool CHK>
__global__ void __launch_bounds__(WX *H, 1)
    k_fused3d_reg(const Args<T> A, Geo g, const Scal *sc, DevInfo *di, int kz) {
  if (di != nullptr && *(volatile const int *)&di->done != 0) return;
  const bool frozen = di != nullptr && di->frozen;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int i0 = blockIdx.x * OX, j0 = blockIdx.y * (H - 4);
  const bool interior = i0 - 2 >= 1 && i0 + WX - 3 <= g.nx - 1 && j0 - 2 >= 1 && j0 + H - 3 <= g.ny - 1;
  if (interior) reg_body<T, H, true, Off, CHK>(A, g, sc, di, frozen, kz, smem_raw);
  else reg_body<T, H, false, Off, CHK>(A, g, sc, di, frozen, kz, smem_raw);
}

template <typename T>
constexpr int reg_rows() { return sizeof(T) == 4 ? 16 : 8; }

}  // namespace

// One fused iteration, register z-march flavour: reads buffer b of the
// stage, writes 1 - b.  check (FP32 only): a check iteration, which also
// reduces the stopping measures into di and updates the check snapshots.
template <typename T>
void launch_fused3d_reg(const Geo &g, const Stage<T> &S, const Scal *sc, DevInfo *di, int kz, cudaStream_t st,
                        bool check) {
  constexpr int H = reg_rows<T>();
  Args<T> A;
  for (int d = 0; d < 3; ++d) {
    A.u[d] = S.u[d]; A.rq[d] = S.rq[d]; A.son[d] = S.son[d]; A.sos[d] = S.sos[d];
    A.tbn[d] = S.tbn[d]; A.tbs[d] = S.tbs[d];
    A.snn[d] = S.snn[d]; A.sns[d] = S.sns[d]; A.uo[d] = S.uo[d];
    A.cn[d] = S.cn[d]; A.cs[d] = S.cs[d]; A.uchk[d] = S.uchk[d]; A.v0[d] = S.v0[d];
  }
  A.rd[0] = S.rd[0]; A.rd[1] = S.rd[1];
  A.sop = S.sop; A.pb = S.pb; A.yc = S.yc; A.snp = S.snp;
  A.s = S.s; A.cp = S.cp;
  kz = fused3d_kz(g, OX, H - 4, kz);
  dim3 grid((g.px + OX - 1) / OX, (g.py + H - 5) / (H - 4), (g.pz + kz - 1) / kz);
  const size_t sm = sizeof(SmemR<T, H>), smc = sm + sizeof(ChkSlots<T, H>);
  if constexpr (sizeof(T) == 4) {
    const bool o32 = (long long)g.pz * g.plane < (1LL << 31);
    if (check) {
      if (o32) k_fused3d_reg<T, H, int, true><<<grid, WX * H, smc, st>>>(A, g, sc, di, kz);
      else k_fused3d_reg<T, H, long long, true><<<grid, WX * H, smc, st>>>(A, g, sc, di, kz);
    } else {
      if (o32) k_fused3d_reg<T, H, int, false><<<grid, WX * H, sm, st>>>(A, g, sc, di, kz);
      else k_fused3d_reg<T, H, long long, false><<<grid, WX * H, sm, st>>>(A, g, sc, di, kz);
    }
  } else {
    k_fused3d_reg<T, H, long long, false><<<grid, WX * H, sm, st>>>(A, g, sc, di, kz);
  }
}

cudaError_t fused3d_reg_configure() {
  const int sf = (int)sizeof(SmemR<float, 16>), sfc = sf + (int)sizeof(ChkSlots<float, 16>);
  cudaError_t e = cudaFuncSetAttribute(k_fused3d_reg<float, 16, int, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, sf);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fused3d_reg<float, 16, long long, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             sf);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fused3d_reg<float, 16, int, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sfc);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fused3d_reg<float, 16, long long, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             sfc);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fused3d_reg<double, 8, long long, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(SmemR<double, 8>));
}

template void launch_fused3d_reg<float>(const Geo &, const Stage<float> &, const Scal *, DevInfo *, int, cudaStream_t,
                                        bool);
template void launch_fused3d_reg<double>(const Geo &, const Stage<double> &, const Scal *, DevInfo *, int,
                                         cudaStream_t, bool);

}  // namespace ep
