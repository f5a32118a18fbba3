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
  double KDt;          // K dt (Eq. A2ssP)
  double A, B;         // Drucker-Prager coefficients (Eqs. A61 / A611)
  double vstep;        // pseudo step / rho~ (Eq. A22P)
  double dt;
  double tol;
  double inv_1mbt, inv_1mbp;  // 1/(1-beta_tau), 1/(1-beta_p)
  double dxmin;
  double rate[3];
  long long n_chk;
  int jaumann;
};

// Reduction slots: bit patterns of non-negative doubles reduced with an
// unsigned atomicMax (IEEE order equals integer order for x >= 0; a NaN
// compares above +inf and so surfaces as "diverged").
enum { RED_R = 0, RED_SIG, RED_DTAU, RED_DP, RED_DU, RED_V, RED_COUNT = 8 };

struct DevInfo {
  unsigned long long red[RED_COUNT];
  int done;            // 0 running, 1 converged, 2 diverged, 3 reached max_iter
  int pad;
  long long k_check;   // iteration index of the next residual check
  long long max_iter;
  long long iters;     // index of the last check taken
  double eps_res, eps_mom, eps_tau, eps_p, eps_rel, max_r, max_sig;
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
  double tb_scale;
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
};

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

// ---- increment set-up and commit (FP64; ep_increment.cu) ------------------
struct History {
  double *v[3], *tn[3], *ts[3], *p, *coh, *epl, *u[3], *an[3], *as[3], *v0[3];
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
void launch_pack(const double *box, double *dst, int ex, int ey, int ez, int px, int py, cudaStream_t st);
void launch_unpack(const double *src, double *box, int ex, int ey, int ez, int px, int py, cudaStream_t st);

}  // namespace ep
