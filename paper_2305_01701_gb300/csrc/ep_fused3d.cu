// ep_fused3d.cu -- one pseudo-transient iteration in one kernel (3D).
//
// The five stages of ep_stages.cu (spin, relaxed trial, centre return, edge
// return, velocity update; Eqs. A5, A23ssP, A2ssP, A6121lambda, A22S, A22P)
// are fused so that each iteration reads every input array once and writes
// the new state once.  A CTA owns a TX x TY column of cells and marches up
// through z one plane per step with a 2-cell halo in x and y:
//   step t loads plane t (prefetched with cp.async during step t-1), then
//     spin/strain of plane t  ->  trials of face-plane t and plane t-1
//     ->  return of plane t-1  ->  new edge deviators (plane t-1)
//     ->  residual and velocity update of plane t-2.
// Halo cells are recomputed by neighbouring CTAs; only the tile's own
// positions are written.  Planes live in shared-memory rings indexed by
// plane mod ring length.  Check iterations (residual norms) stay on the
// staged kernels.
#include <math.h>

#include "ep_internal.cuh"

namespace ep {

namespace {

constexpr int TX = 32;

// ring lengths
constexpr int RU = 4;   // velocity increment planes t-2 .. t (+1 in flight)
constexpr int RC = 3;   // rotation weights planes t-1, t (+1 in flight)

template <typename T, int TY>
struct Smem {
  static constexpr int W = TX + 4, H = TY + 4, WH = W * H;
  T vx[RU][WH], vy[RU][WH], vz[RU][WH];
  T rqxy[RC][WH], rqxz[RC][WH], rqyz[RC][WH], rd0[RC][WH], rd1[RC][WH];
  T oxy[2][WH], oxz[2][WH], oyz[2][WH];
  T exy[2][WH], exz[WH], eyz[WH];
  T txy[WH], txz[2][WH], tyz[2][WH], tc[3][WH];
  T s[2][WH];
  T sxx[2][WH], syy[2][WH], szz[3][WH];
  T nxy[2][WH], nxz[2][WH], nyz[2][WH];
};

__device__ __forceinline__ int rs(int lev, int R) { return ((lev % R) + R) % R; }

__device__ __forceinline__ void cp_async_el(float *smem, const float *gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_el(double *smem, const double *gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

template <typename T>
struct F3 {
  const T *u[3];
  const T *son[3], *sos[3], *sop;
  T *snn[3], *sns[3], *snp;
  const T *tbn[3], *tbs[3], *pb, *yc;
  const T *rq[3], *rd[2];
  T *uo[3];
  const T *s;   // centre return scales (read when plasticity is frozen)
};

// Load plane `lev` of the neighbour-read inputs into their ring slots.
// Positions outside the padded box or the plane range read as zero.
template <typename T, int TY>
__device__ __forceinline__ void load_plane(Smem<T, TY> &S, const F3<T> &A, const Geo &g, int i0, int j0, int lev) {
  constexpr int W = Smem<T, TY>::W, WH = Smem<T, TY>::WH, NT = TX * TY;
  const int su = rs(lev, RU), sc = rs(lev, RC);
  const bool lev_ok = lev >= 0 && lev < g.pz;
  for (int p = threadIdx.x; p < WH; p += NT) {
    const int a = p % W, b = p / W;
    const int gi = i0 - 2 + a, gj = j0 - 2 + b;
    const bool ok = lev_ok && gi >= 0 && gi < g.px && gj >= 0 && gj < g.py;
    if (ok) {
      const long long e = ((long long)lev * g.py + gj) * g.px + gi;
      cp_async_el(&S.vx[su][p], A.u[0] + e);
      cp_async_el(&S.vy[su][p], A.u[1] + e);
      cp_async_el(&S.vz[su][p], A.u[2] + e);
      cp_async_el(&S.rqxy[sc][p], A.rq[0] + e);
      cp_async_el(&S.rqxz[sc][p], A.rq[1] + e);
      cp_async_el(&S.rqyz[sc][p], A.rq[2] + e);
      cp_async_el(&S.rd0[sc][p], A.rd[0] + e);
      cp_async_el(&S.rd1[sc][p], A.rd[1] + e);
    } else {
      S.vx[su][p] = (T)0; S.vy[su][p] = (T)0; S.vz[su][p] = (T)0;
      S.rqxy[sc][p] = (T)0; S.rqxz[sc][p] = (T)0; S.rqyz[sc][p] = (T)0;
      S.rd0[sc][p] = (T)0; S.rd1[sc][p] = (T)0;
    }
  }
}

template <typename T, int TY>
__global__ void __launch_bounds__(TX * TY, 2) k_fused3d(Geo g, F3<T> A, const Scal *sc, const DevInfo *di, int kz) {
  constexpr int W = Smem<T, TY>::W, H = Smem<T, TY>::H, WH = Smem<T, TY>::WH, NT = TX * TY;
  if (di != nullptr && *(volatile const int *)&di->done != 0) return;
  const bool frozen = di != nullptr && di->frozen;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T, TY> &S = *reinterpret_cast<Smem<T, TY> *>(smem_raw);
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int kb = blockIdx.z * kz, ke = min(kb + kz, g.pz);
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const T rdx = (T)g.rdx, rdy = (T)g.rdy, rdz = (T)g.rdz;
  const T two_eta = (T)sc->two_eta, bt = (T)sc->bt, ob = (T)1 - bt;
  const T bp = (T)sc->bp, obp = (T)sc->obp, KDt = (T)sc->KDt, Acoef = (T)sc->A;
  const T vs = (T)sc->vstep, qr = (T)0.25, third = (T)(1.0 / 3.0);
  const long long px = g.px;

  // clear the rings that are read before first written (planes below kb-2)
  for (int p = threadIdx.x; p < WH; p += NT) {
#pragma unroll
    for (int r = 0; r < RU; ++r) { S.vx[r][p] = (T)0; S.vy[r][p] = (T)0; S.vz[r][p] = (T)0; }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      S.oxy[r][p] = (T)0; S.oxz[r][p] = (T)0; S.oyz[r][p] = (T)0; S.exy[r][p] = (T)0;
      S.txz[r][p] = (T)0; S.tyz[r][p] = (T)0; S.s[r][p] = (T)0; S.sxx[r][p] = (T)0; S.syy[r][p] = (T)0;
      S.nxy[r][p] = (T)0; S.nxz[r][p] = (T)0; S.nyz[r][p] = (T)0;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) S.szz[r][p] = (T)0;
  }
  __syncthreads();
  load_plane(S, A, g, i0, j0, kb - 2);
  cp_async_commit();

  for (int t = kb - 2; t < ke + 2; ++t) {
    cp_async_wait_all();
    __syncthreads();
    load_plane(S, A, g, i0, j0, t + 1);
    cp_async_commit();

    const int u0 = rs(t, RU), um1 = rs(t - 1, RU), um2 = rs(t - 2, RU);
    const int c0 = rs(t, RC), cm1 = rs(t - 1, RC);
    const int o0 = rs(t, 2), om1 = rs(t - 1, 2), om2 = rs(t - 2, 2);

    // ---- 1. shear strain rate and spin: xy plane t, xz/yz face-plane t ----
    for (int p = threadIdx.x; p < WH; p += NT) {
      const int a = p % W, b = p / W;
      const int gi = i0 - 2 + a, gj = j0 - 2 + b;
      T es = (T)0, om = (T)0;
      if (a >= 1 && b >= 1 && t >= 0 && t < nz && gi >= 1 && gi <= nx - 1 && gj >= 1 && gj <= ny - 1) {
        T x = (S.vx[u0][p] - S.vx[u0][p - W]) * rdy;   // dvx/dy
        T y = (S.vy[u0][p] - S.vy[u0][p - 1]) * rdx;   // dvy/dx
        es = (T)0.5 * (x + y); om = (T)0.5 * (x - y);
      }
      S.exy[o0][p] = es; S.oxy[o0][p] = om;
      es = (T)0; om = (T)0;
      if (a >= 1 && t >= 1 && t <= nz - 1 && gi >= 1 && gi <= nx - 1 && gj >= 0 && gj < ny) {
        T x = (S.vx[u0][p] - S.vx[um1][p]) * rdz;      // dvx/dz
        T y = (S.vz[u0][p] - S.vz[u0][p - 1]) * rdx;   // dvz/dx
        es = (T)0.5 * (x + y); om = (T)0.5 * (x - y);
      }
      S.exz[p] = es; S.oxz[o0][p] = om;
      es = (T)0; om = (T)0;
      if (b >= 1 && t >= 1 && t <= nz - 1 && gi >= 0 && gi < nx && gj >= 1 && gj <= ny - 1) {
        T x = (S.vy[u0][p] - S.vy[um1][p]) * rdz;      // dvy/dz
        T y = (S.vz[u0][p] - S.vz[u0][p - W]) * rdy;   // dvz/dy
        es = (T)0.5 * (x + y); om = (T)0.5 * (x - y);
      }
      S.eyz[p] = es; S.oyz[o0][p] = om;
    }
    __syncthreads();

    // ---- 2. relaxed trials: xz/yz face-plane t, xy and centres plane t-1 ----
    const int lc = t - 1;  // centre plane of this step's return
    for (int p = threadIdx.x; p < WH; p += NT) {
      const int a = p % W, b = p / W;
      const int gi = i0 - 2 + a, gj = j0 - 2 + b;
      const long long ef = ((long long)t * g.py + gj) * px + gi;     // face-plane t
      const long long ec = ((long long)lc * g.py + gj) * px + gi;    // plane t-1
      // xz-edge (x_i, yc_j, z_t)
      T v = (T)0;
      if (a >= 1 && b < H - 1 && t >= 1 && t <= nz - 1 && gi >= 1 && gi <= nx - 1 && gj >= 0 && gj < ny) {
        T dzx = qr * (S.rd1[cm1][p - 1] + S.rd1[cm1][p] + S.rd1[c0][p - 1] + S.rd1[c0][p]);
        T Tyz = qr * (S.rqyz[c0][p - 1] + S.rqyz[c0][p] + S.rqyz[c0][p - 1 + W] + S.rqyz[c0][p + W]);
        T Wyz = qr * (S.oyz[o0][p - 1] + S.oyz[o0][p] + S.oyz[o0][p - 1 + W] + S.oyz[o0][p + W]);
        T Txy = qr * (S.rqxy[cm1][p] + S.rqxy[cm1][p + W] + S.rqxy[c0][p] + S.rqxy[c0][p + W]);
        T Wxy = qr * (S.oxy[om1][p] + S.oxy[om1][p + W] + S.oxy[o0][p] + S.oxy[o0][p + W]);
        T tr = A.tbs[1][ef] + two_eta * S.exz[p] + (S.oxz[o0][p] * dzx + Tyz * Wxy - Txy * Wyz);
        v = bt * A.sos[1][ef] + ob * tr;
      }
      S.txz[o0][p] = v;
      // yz-edge (xc_i, y_j, z_t)
      v = (T)0;
      if (a < W - 1 && b >= 1 && t >= 1 && t <= nz - 1 && gi >= 0 && gi < nx && gj >= 1 && gj <= ny - 1) {
        T dzy = qr * ((S.rd1[cm1][p - W] - S.rd0[cm1][p - W]) + (S.rd1[cm1][p] - S.rd0[cm1][p]) +
                          (S.rd1[c0][p - W] - S.rd0[c0][p - W]) + (S.rd1[c0][p] - S.rd0[c0][p]));
        T Txy = qr * (S.rqxy[cm1][p] + S.rqxy[cm1][p + 1] + S.rqxy[c0][p] + S.rqxy[c0][p + 1]);
        T Wxy = qr * (S.oxy[om1][p] + S.oxy[om1][p + 1] + S.oxy[o0][p] + S.oxy[o0][p + 1]);
        T Txz = qr * (S.rqxz[c0][p - W] + S.rqxz[c0][p - W + 1] + S.rqxz[c0][p] + S.rqxz[c0][p + 1]);
        T Wxz = qr * (S.oxz[o0][p - W] + S.oxz[o0][p - W + 1] + S.oxz[o0][p] + S.oxz[o0][p + 1]);
        T tr = A.tbs[2][ef] + two_eta * S.eyz[p] + (S.oyz[o0][p] * dzy - Txy * Wxz - Txz * Wxy);
        v = bt * A.sos[2][ef] + ob * tr;
      }
      S.tyz[o0][p] = v;
      // xy-edge (x_i, y_j, zc_{t-1})
      v = (T)0;
      if (a >= 1 && b >= 1 && lc >= 0 && lc < nz && gi >= 1 && gi <= nx - 1 && gj >= 1 && gj <= ny - 1) {
        T dyx = qr * (S.rd0[cm1][p - W - 1] + S.rd0[cm1][p - W] + S.rd0[cm1][p - 1] + S.rd0[cm1][p]);
        T Tyz = qr * (S.rqyz[cm1][p - 1] + S.rqyz[cm1][p] + S.rqyz[c0][p - 1] + S.rqyz[c0][p]);
        T Wyz = qr * (S.oyz[om1][p - 1] + S.oyz[om1][p] + S.oyz[o0][p - 1] + S.oyz[o0][p]);
        T Txz = qr * (S.rqxz[cm1][p - W] + S.rqxz[cm1][p] + S.rqxz[c0][p - W] + S.rqxz[c0][p]);
        T Wxz = qr * (S.oxz[om1][p - W] + S.oxz[om1][p] + S.oxz[o0][p - W] + S.oxz[o0][p]);
        T tr = A.tbs[0][ec] + two_eta * S.exy[om1][p] + (S.oxy[om1][p] * dyx + Tyz * Wxz + Txz * Wyz);
        v = bt * A.sos[0][ec] + ob * tr;
      }
      S.txy[p] = v;
      // centre (xc_i, yc_j, zc_{t-1})
      if (a < W - 1 && b < H - 1 && lc >= 0 && lc < nz && gi >= 0 && gi < nx && gj >= 0 && gj < ny) {
        T exx = (S.vx[um1][p + 1] - S.vx[um1][p]) * rdx;
        T eyy = (S.vy[um1][p + W] - S.vy[um1][p]) * rdy;
        T ezz = (S.vz[u0][p] - S.vz[um1][p]) * rdz;
        T d3 = (exx + eyy + ezz) * third;
        T pxy = qr * (S.rqxy[cm1][p] * S.oxy[om1][p] + S.rqxy[cm1][p + 1] * S.oxy[om1][p + 1] +
                          S.rqxy[cm1][p + W] * S.oxy[om1][p + W] + S.rqxy[cm1][p + W + 1] * S.oxy[om1][p + W + 1]);
        T pxz = qr * (S.rqxz[cm1][p] * S.oxz[om1][p] + S.rqxz[cm1][p + 1] * S.oxz[om1][p + 1] +
                          S.rqxz[c0][p] * S.oxz[o0][p] + S.rqxz[c0][p + 1] * S.oxz[o0][p + 1]);
        T pyz = qr * (S.rqyz[cm1][p] * S.oyz[om1][p] + S.rqyz[cm1][p + W] * S.oyz[om1][p + W] +
                          S.rqyz[c0][p] * S.oyz[o0][p] + S.rqyz[c0][p + W] * S.oyz[o0][p + W]);
        T t0 = A.tbn[0][ec] + two_eta * (exx - d3) + (T)2 * (pxy + pxz);
        T t1 = A.tbn[1][ec] + two_eta * (eyy - d3) - (T)2 * (pxy - pyz);
        T t2 = A.tbn[2][ec] + two_eta * (ezz - d3) - (T)2 * (pxz + pyz);
        S.tc[0][p] = bt * A.son[0][ec] + ob * t0;
        S.tc[1][p] = bt * A.son[1][ec] + ob * t1;
        S.tc[2][p] = bt * A.son[2][ec] + ob * t2;
      } else {
        S.tc[0][p] = (T)0; S.tc[1][p] = (T)0; S.tc[2][p] = (T)0;
      }
    }
    __syncthreads();

    // ---- 3. pressure and return at centres of plane t-1 ----
    const int s1 = rs(lc, 2), z1 = rs(lc, 3);
    for (int p = threadIdx.x; p < WH; p += NT) {
      const int a = p % W, b = p / W;
      const int gi = i0 - 2 + a, gj = j0 - 2 + b;
      T s = (T)0, sx = (T)0, sy = (T)0, sz = (T)0;
      if (a >= 1 && a < W - 1 && b >= 1 && b < H - 1 && lc >= 0 && lc < nz && gi >= 0 && gi < nx && gj >= 0 &&
          gj < ny) {
        const long long ec = ((long long)lc * g.py + gj) * px + gi;
        T div = (S.vx[um1][p + 1] - S.vx[um1][p]) * rdx + (S.vy[um1][p + W] - S.vy[um1][p]) * rdy +
                    (S.vz[u0][p] - S.vz[um1][p]) * rdz;
        T pr = bp * A.sop[ec] + obp * (A.pb[ec] - KDt * div);
        T txy = qr * (S.txy[p] + S.txy[p + 1] + S.txy[p + W] + S.txy[p + W + 1]);
        T txz = qr * (S.txz[om1][p] + S.txz[om1][p + 1] + S.txz[o0][p] + S.txz[o0][p + 1]);
        T tyz = qr * (S.tyz[om1][p] + S.tyz[om1][p + W] + S.tyz[o0][p] + S.tyz[o0][p + W]);
        T T0 = S.tc[0][p], T1 = S.tc[1][p], T2 = S.tc[2][p];
        T J2 = txy * txy + txz * txz + tyz * tyz + (T)0.5 * T0 * T0 + (T)0.5 * T1 * T1 + (T)0.5 * T2 * T2;
        if (frozen) {
          s = A.s[ec];
        } else {
          T sj = sqrt(J2);
          T Y = Acoef * pr + A.yc[ec];
          Y = Y > (T)0 ? Y : (T)0;
          s = sj > Y ? Y / sj : (T)1;
        }
        T n0 = s * T0, n1 = s * T1, n2 = s * T2;
        sx = n0 - pr; sy = n1 - pr; sz = n2 - pr;
        if (a >= 2 && a < W - 2 && b >= 2 && b < H - 2 && lc >= kb && lc < ke) {
          A.snn[0][ec] = n0; A.snn[1][ec] = n1; A.snn[2][ec] = n2; A.snp[ec] = pr;
        }
      }
      S.s[s1][p] = s; S.sxx[s1][p] = sx; S.syy[s1][p] = sy; S.szz[z1][p] = sz;
    }
    __syncthreads();

    // ---- 4. new edge deviators: xy plane t-1, xz/yz face-plane t-1 ----
    const int sm2 = rs(lc - 1, 2);
    for (int p = threadIdx.x; p < WH; p += NT) {
      const int a = p % W, b = p / W;
      const int gi = i0 - 2 + a, gj = j0 - 2 + b;
      T vxy = (T)0, vxz = (T)0, vyz = (T)0;
      const bool inner = a >= 2 && a < W - 1 && b >= 2 && b < H - 1;
      if (inner && lc >= 0 && lc < nz && gi >= 1 && gi <= nx - 1 && gj >= 1 && gj <= ny - 1)
        vxy = qr * (S.s[s1][p - W - 1] + S.s[s1][p - W] + S.s[s1][p - 1] + S.s[s1][p]) * S.txy[p];
      if (inner && lc >= 1 && lc <= nz - 1 && gi >= 1 && gi <= nx - 1 && gj >= 0 && gj < ny)
        vxz = qr * (S.s[sm2][p - 1] + S.s[sm2][p] + S.s[s1][p - 1] + S.s[s1][p]) * S.txz[om1][p];
      if (inner && lc >= 1 && lc <= nz - 1 && gi >= 0 && gi < nx && gj >= 1 && gj <= ny - 1)
        vyz = qr * (S.s[sm2][p - W] + S.s[sm2][p] + S.s[s1][p - W] + S.s[s1][p]) * S.tyz[om1][p];
      S.nxy[s1][p] = vxy; S.nxz[s1][p] = vxz; S.nyz[s1][p] = vyz;
      if (a >= 2 && a < W - 2 && b >= 2 && b < H - 2 && lc >= kb && lc < ke && gi < g.px && gj < g.py) {
        const long long e = ((long long)lc * g.py + gj) * px + gi;
        A.sns[0][e] = vxy; A.sns[1][e] = vxz; A.sns[2][e] = vyz;
      }
    }
    __syncthreads();

    // ---- 5. residual and velocity update of plane t-2 ----
    const int lu = t - 2;
    if (lu >= kb && lu < ke) {
      const int q2 = rs(lu, 2), q1 = rs(lu + 1, 2), z2 = rs(lu, 3), z3 = rs(lu - 1, 3);
      for (int p = threadIdx.x; p < NT; p += NT) {
        const int a = 2 + p % TX, b = 2 + p / TX, pp = b * W + a;
        const int gi = i0 + p % TX, gj = j0 + p / TX;
        if (gi >= g.px || gj >= g.py) continue;
        const long long e = ((long long)lu * g.py + gj) * px + gi;
        // x-face
        T u = S.vx[um2][pp], un = u;
        if (gi >= 1 && gi <= nx - 1 && gj < ny && lu < nz) {
          T R = (S.sxx[q2][pp] - S.sxx[q2][pp - 1]) * rdx + (S.nxy[q2][pp + W] - S.nxy[q2][pp]) * rdy +
                    (S.nxz[q1][pp] - S.nxz[q2][pp]) * rdz;
          un = u + vs * R;
        }
        A.uo[0][e] = un;
        // y-face
        u = S.vy[um2][pp]; un = u;
        if (gj >= 1 && gj <= ny - 1 && gi < nx && lu < nz) {
          T R = (S.syy[q2][pp] - S.syy[q2][pp - W]) * rdy + (S.nxy[q2][pp + 1] - S.nxy[q2][pp]) * rdx +
                    (S.nyz[q1][pp] - S.nyz[q2][pp]) * rdz;
          un = u + vs * R;
        }
        A.uo[1][e] = un;
        // z-face
        u = S.vz[um2][pp]; un = u;
        if (lu >= 1 && lu <= nz - 1 && gi < nx && gj < ny) {
          T R = (S.szz[z2][pp] - S.szz[z3][pp]) * rdz + (S.nxz[q2][pp + 1] - S.nxz[q2][pp]) * rdx +
                    (S.nyz[q2][pp + W] - S.nyz[q2][pp]) * rdy;
          un = u + vs * R;
        }
        A.uo[2][e] = un;
      }
    }
  }
  cp_async_wait_all();
}

}  // namespace

template <typename T>
constexpr int fused_ty() { return sizeof(T) == 4 ? 8 : 4; }

template <typename T>
size_t fused3d_smem_bytes() { return sizeof(Smem<T, fused_ty<T>()>); }

// One fused iteration: reads buffer b of the stage, writes 1 - b.
template <typename T>
void launch_fused3d(const Geo &g, const Stage<T> &S, const Scal *sc, const DevInfo *di, int kz, cudaStream_t st) {
  constexpr int TY = fused_ty<T>();
  F3<T> A;
  for (int d = 0; d < 3; ++d) {
    A.u[d] = S.u[d]; A.son[d] = S.son[d]; A.sos[d] = S.sos[d]; A.snn[d] = S.snn[d]; A.sns[d] = S.sns[d];
    A.tbn[d] = S.tbn[d]; A.tbs[d] = S.tbs[d]; A.rq[d] = S.rq[d]; A.uo[d] = S.uo[d];
  }
  A.sop = S.sop; A.snp = S.snp; A.pb = S.pb; A.yc = S.yc; A.rd[0] = S.rd[0]; A.rd[1] = S.rd[1];
  A.s = S.s;
  kz = fused3d_kz(g, TX, TY, kz, 2);
  dim3 grid((g.px + TX - 1) / TX, (g.py + TY - 1) / TY, (g.pz + kz - 1) / kz);
  k_fused3d<T, TY><<<grid, TX * TY, sizeof(Smem<T, TY>), st>>>(g, A, sc, di, kz);
}

cudaError_t fused3d_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_fused3d<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(Smem<float, 8>));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fused3d<double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(Smem<double, 4>));
}

template size_t fused3d_smem_bytes<float>();
template size_t fused3d_smem_bytes<double>();
template void launch_fused3d<float>(const Geo &, const Stage<float> &, const Scal *, const DevInfo *, int,
                                    cudaStream_t);
template void launch_fused3d<double>(const Geo &, const Stage<double> &, const Scal *, const DevInfo *, int,
                                     cudaStream_t);

}  // namespace ep
