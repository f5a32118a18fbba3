// ep_internal.cuh -- device-side data layout and kernel interfaces of libep.
//
// Layout in HBM: every field of a grid lives in one padded box of
// px x py x pz elements, x fastest, px a multiple of 32 (coalesced, 128-byte
// aligned rows), py = ny + 1, pz = nz + 1 (3D) or 1 (2D).  All staggered
// locations share that box and its index (i, j, k) -> (k py + j) px + i:
// centre (i,j,k), x-face i at x_i, vertex/edge (i,j,k) at the lower corner.
// Positions outside a location's extent are kept at zero.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ep.h"

namespace ep {

struct Geo {
  int ndim, nx, ny, nz;
  int px, py, pz;
  long long plane, box;
  double dx, dy, dz, rdx, rdy, rdz;
  __host__ __device__ __forceinline__ long long idx(int i, int j, int k) const {
    return ((long long)k * py + j) * px + i;
  }
};

// Per-increment scalars, read by the kernels from device memory so that a
// captured CUDA graph stays valid across increments.
struct Scal {
  double two_eta;      // 2 eta_ve
  double c2;           // eta_ve / (G dt): weight of the rotated old stress
  double c2dt;         // c2 * dt: weight of the Jaumann rotation term
  double bt, bp;       // relaxation weights beta_tau, beta_p (Eqs. A23ssP, A2ssP)
  double KDt;          // sweep pressure step: K dt (Eq. A2ssP), K~ incompressible (Eq. A2ssP2)
  double obp;          // weight of the pressure target: 1 - beta_p; 1 incompressible
  double KDt_phys;     // physical response: K dt; 0 incompressible (p stays p_hat)
  double p_meas;       // pressure measure factor: 1 / (1 - beta_p); 2 eta_ve / K~ incompressible
  double A, B;         // Drucker-Prager coefficients (Eqs. A61 / A611)
  double vstep;        // pseudo step / rho~ (Eq. A22P)
  double dt;
  double tol;
  double inv_1mbt, inv_1mbp;  // 1/(1-beta_tau), 1/(1-beta_p)
  double dxmin;
  double rate[3];
  long long n_chk;
  int jaumann;
  long long freeze_iter;   // > 0: frozen plasticity armed from this iteration on
  double freeze_eps;
  long long wait_cycles;   // bound of a TMA wait (0: the default, 2^31 cycles)
  int gcell;               // 1: per-cell shear modulus; the rotation weights then
                           // carry dt only and the trial applies each point's c2
};

// Reduction slots: bit patterns of non-negative doubles reduced with an
// unsigned atomicMax (IEEE order equals integer order for x >= 0; a NaN
// compares above +inf and so surfaces as "diverged").
enum { RED_R = 0, RED_SIG, RED_DTAU, RED_DP, RED_DU, RED_V, RED_COUNT = 8 };

struct DevInfo {
  unsigned long long red[RED_COUNT];
  int done;            // 0 running, 1 converged, 2 diverged, 3 reached max_iter
  int frozen;          // 1: the centre return scales are held (Sec. 3.3)
  long long k_check;   // iteration index of the next residual check
  long long max_iter;
  long long iters;     // index of the last check taken
  double eps_res, eps_mom, eps_tau, eps_p, eps_rel, max_r, max_sig;
  long long frozen_at; // check at which the scales froze, -1 if not
};

// Pointers of one stage evaluation.  The same kernels serve the FP64
// start-of-increment and commit passes (u = full velocity, beta = 0) and the
// sweeps (u = velocity increment, beta from Scal).
template <typename T>
struct Stage {
  const T *u[3];                    // velocity-like face field
  const T *son[3], *sos[3], *sop;   // old pseudo-time state (relax only)
  T *snn[3], *sns[3], *snp;         // new state
  const T *tbn[3], *tbs[3], *pb;    // base trial (x tb_scale) and base pressure
  double tb_scale;                  // 0 with per-cell c2 (then c2 of the point, see tb_c2)
  int tb_c2;                        // 1: the base trial is the old stress times c2
  const T *rq[3];                   // c2 dt tau_hat shear (edges)
  const T *rd[2];                   // c2 dt (tyy - txx), c2 dt (tzz - txx) (centres)
  const T *yc;                      // B c (centres)
  T *om[3], *es[3];                 // spin and shear strain rate of u (edges)
  T *Tn[3], *Ts[3];                 // relaxed trial
  T *s;                             // centre return scale
  T *uo[3];                         // updated face field
  const T *f[3];                    // body force (nullable)
  T *uchk[3];                       // snapshot for eps_rel (check iterations)
  T *cn[3], *cs[3], *cp;            // stress state at the previous check
  const double *v0[3];              // start velocity (eps_rel)
  int relax;                        // 1: sweep weights; 0: physical response
  // per-cell shear modulus (nullable: the uniform scalars): 2 eta_ve and
  // c2 = eta_ve / (G dt) at centres [0] and vertices/edges [1 + c]
  const T *ge[4], *gc[4];
};

// One 2D instance of the batched fused sweep (ep_fused2d.cu): geometry,
// scalars, convergence record and both ping-pong buffers of every array.
template <typename T>
struct Inst2 {
  Geo g;
  const Scal *sc;
  DevInfo *di;
  T *u[2][2];                       // [buffer][component]
  T *sn[2][2], *ss[2], *sp[2];      // stress state: centres [buffer][comp], vertices, pressure
  const T *tbn[2], *tbs, *pb, *yc, *rq, *rd;
  T *s;
  T *uchk[2], *cn[2], *cs, *cp;
  const double *v0[2];
};

// Convergence decision after a check iteration (Eqs. Convergence1-3 in the
// stopping measures described in ep_stages.cu).
__device__ __forceinline__ void check_one(DevInfo *di, const Scal *sc) {
  if (di->done) return;
  auto bits = [](unsigned long long b) { return __longlong_as_double((long long)b); };
  const double mr = bits(di->red[RED_R]), ms = bits(di->red[RED_SIG]);
  const double dtau = bits(di->red[RED_DTAU]), dp = bits(di->red[RED_DP]);
  const double du = bits(di->red[RED_DU]), vm = bits(di->red[RED_V]);
  const double inf = __longlong_as_double(0x7ff0000000000000ll);
  // iterations since the previous check (the start state for the first one)
  const double m = di->k_check == 0 ? 1.0 : (double)sc->n_chk;
  // momentum residual averaged over the interval: rho~ (u_{k+1} - u_chk) / m
  double em = du == 0.0 ? 0.0 : (ms > 0.0 ? sc->dxmin * du / (m * sc->vstep) / ms : inf);
  double et = dtau == 0.0 ? 0.0 : (ms > 0.0 ? dtau / (m * (1.0 - sc->bt)) / ms : inf);
  double ep = dp == 0.0 ? 0.0 : (ms > 0.0 ? dp * sc->p_meas / m / ms : inf);
  double er = em > et ? em : et;
  if (ep > er) er = ep;
  if (isnan(em) || isnan(et) || isnan(ep) || isnan(ms) || isnan(du)) er = nan("");
  const long long k = di->k_check;
  di->iters = k;
  di->eps_res = er; di->eps_mom = em; di->eps_tau = et; di->eps_p = ep;
  di->eps_rel = vm > 0.0 ? du / vm : 0.0;
  di->max_r = mr; di->max_sig = ms;
  if (isnan(er) || isnan(mr) || isnan(du)) di->done = 2;
  else if (er <= sc->tol) di->done = 1;
  else if (k >= di->max_iter) di->done = 3;
  else {
    di->k_check = k + sc->n_chk;
    // frozen plasticity (Sec. 3.3): hold the scales of this check iteration
    if (!di->frozen && sc->freeze_iter > 0 && k >= sc->freeze_iter && di->eps_rel > sc->freeze_eps) {
      di->frozen = 1;
      di->frozen_at = k;
    }
  }
  for (int r = 0; r < RED_COUNT; ++r) di->red[r] = 0ull;
}

// ---- batched fused 2D sweep (ep_fused2d.cu, ep_fused2d_strip.cu) ---------
// tile: 0 = 32x8, 1 = 32x16, 2 = 64x8 cells (block tiles in shared memory);
// 3, 4 = warp strips of 28 columns marching 64 / 32 rows
constexpr int FUSED2D_TILES = 5;
inline int fused2d_items_per_block(int tile) { return tile >= 3 ? 8 : 1; }
template <typename T>
void launch_fused2d_strip(int seg, const Inst2<T> *insts, const int4 *items, int n_items, int b, int check,
                          int blocks, cudaStream_t st);
template <typename T>
int fused2d_strip_blocks_per_sm(int seg);
template <typename T>
void launch_fused2d(int tile, const Inst2<T> *insts, const int4 *items, int n_items, int b, int check, int blocks,
                    cudaStream_t st);
template <typename T>
void launch_check_batch(const Inst2<T> *insts, int n, cudaStream_t st);
template <typename T>
void launch_init_batch(const Inst2<T> *insts, int n, long long max_iter, cudaStream_t st);
void fused2d_tile(int tile, int *tx, int *ty);
cudaError_t fused2d_configure();
template <typename T>
int fused2d_blocks_per_sm(int tile);

// ---- staged sweep (one kernel per stage; ep_stages.cu) --------------------
template <typename T>
void launch_strain(const Geo &g, const Stage<T> &S, const Scal *sc, DevInfo *di, cudaStream_t st);
template <typename T>
void launch_trial(const Geo &g, const Stage<T> &S, const Scal *sc, DevInfo *di, cudaStream_t st);
template <typename T>
void launch_return_centres(const Geo &g, const Stage<T> &S, const Scal *sc, DevInfo *di, int check,
                           cudaStream_t st);
template <typename T>
void launch_return_edges(const Geo &g, const Stage<T> &S, const Scal *sc, DevInfo *di, int check,
                         cudaStream_t st);
template <typename T>
void launch_velocity(const Geo &g, const Stage<T> &S, const Scal *sc, DevInfo *di, int check,
                     cudaStream_t st);
void launch_check(DevInfo *di, const Scal *sc, cudaStream_t st);

// ---- fused sweeps (ep_fused3d.cu) ------------------------------------
// z-planes per block when none was chosen (kz <= 0).  A block marches kz
// planes plus four halo planes, and the launch runs in waves of
// (SMs x blocks per SM) blocks, so the time goes as
// waves(kz) x (kz + 4); take the kz in [8, 128] that minimises it.
inline int fused3d_kz(const Geo &g, int tx, int ty, int kz, int per_sm = 1) {
  if (kz > 0) return kz;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
  }
  const long long cols = (long long)((g.px + tx - 1) / tx) * ((g.py + ty - 1) / ty);
  const long long wave = (long long)sms * per_sm;
  int best = 8;
  long long best_cost = -1;
  for (int k = 8; k <= 128; ++k) {
    const long long blocks = cols * ((g.pz + k - 1) / k);
    const long long cost = (blocks + wave - 1) / wave * (k + 4);
    if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = k; }
  }
  return best;
}
template <typename T>
size_t fused3d_smem_bytes();
cudaError_t fused3d_configure();
template <typename T>
void launch_fused3d(const Geo &g, const Stage<T> &S, const Scal *sc, const DevInfo *di, int kz, cudaStream_t st);
// TMA-streamed variant (ep_fused3d_tma.cu); false if a tensor map failed
template <typename T>
bool launch_fused3d_tma(const Geo &g, const Stage<T> &S, const Scal *sc, const DevInfo *di, int kz, cudaStream_t st);
cudaError_t fused3d_tma_configure();
// register z-march variant (ep_fused3d_reg.cu)
template <typename T>
void launch_fused3d_reg(const Geo &g, const Stage<T> &S, const Scal *sc, DevInfo *di, int kz, cudaStream_t st,
                        bool check = false);
cudaError_t fused3d_reg_configure();

// ---- increment set-up and commit (FP64; ep_increment.cu) ------------------
struct History {
  double *v[3], *tn[3], *ts[3], *p, *coh, *epl, *u[3], *an[3], *as[3], *v0[3];
  const double *te_c;   // per-cell 2 eta_ve at centres (nullable: Scal.two_eta)
};
void launch_start_velocity(const Geo &g, const History &H, const double *const dv[3], const Scal *sc,
                           int started, const double L[3], cudaStream_t st);
template <typename T>
void launch_rotation_fields(const Geo &g, const History &H, const Scal *sc, T *const rq[3], T *const rd[2],
                            T *yc, cudaStream_t st);
template <typename T>
void launch_compose(const Geo &g, const double *const v0[3], const T *const u[3], double *const out[3],
                    cudaStream_t st);
template <typename T>
void launch_commit(const Geo &g, const History &H, const double *const Tn64[3], const double *const Ts64[3],
                   const double *const es64[3], const T *const stn[3], const T *const sts[3], const T *stp,
                   const T *s, const Scal *sc, unsigned long long *n_plastic, cudaStream_t st);
template <typename Td, typename Ts>
void launch_convert(Td *dst, const Ts *src, long long n, cudaStream_t st);
void launch_line_integrals(const Geo &g, const History &H, double *out2, cudaStream_t st);
void launch_advect(const Geo &g, const History &H, const Scal *sc, double *const tn_out[3], double *const ts_out[3],
                   double *p_out, cudaStream_t st);
void launch_pack(const double *box, double *dst, int ex, int ey, int ez, int px, int py, cudaStream_t st);
// learned warm start (ep_warm.cu): 1 / the scales of the channels
struct WarmScales {
  double sv_inv;    // 1 / S_v, S_v = 0.1 |a| L_max
  double st_inv;    // 1 / S_t, S_t = 2 G |a| dt
  double se_inv;    // 1 / S_e, S_e = 10 |a| dt
  double cmax_inv;  // 1 / max c
};
__host__ __device__ constexpr int warm_in_channels(int nd) { return nd == 3 ? 13 : 9; }
__host__ __device__ constexpr int warm_out_channels(int nd) { return nd == 3 ? 9 : 5; }
template <typename T>
void launch_warm_features(const Geo &g, const History &H, const double *const vp[3], const T *s_last,
                          const WarmScales &ws, int f, float *x, const int dims[3], cudaStream_t st);
void launch_warm_target(const Geo &g, const History &H, const double *const vp[3], const float *w0,
                        const WarmScales &ws, int f, float *out, const int dims[3], cudaStream_t st);
void launch_warm_record(const Geo &g, const double *const n[3], const double *const s[3], float *w0,
                        cudaStream_t st);
void launch_warm_dv(const Geo &g, const float *y, int f, double sv, double *const dv[3], const int dims[3],
                    cudaStream_t st);
void launch_warm_stress(const Geo &g, const float *y, int f, double stress_scale, double *const n[3],
                        double *const s[3], const int dims[3], cudaStream_t st);
void launch_shear_fields(const Geo &g, const double *Gc, double mu_s, double dt, double *const ge[4],
                         double *const gc[4], cudaStream_t st);
void launch_scaled_div(const Geo &g, const double *const v[3], double scale, double *out, cudaStream_t st);
void launch_unpack(const double *src, double *box, int ex, int ey, int ez, int px, int py, cudaStream_t st);

}  // namespace ep
