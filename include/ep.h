/*
 * ep.h -- C ABI of the GB300 pseudo-transient elasto-plastic solver.
 *
 * The library advances a (visco-)hypoelastic, perfectly plastic
 * Drucker-Prager medium on a conservative staggered grid, one load increment
 * at a time, with the accelerated pseudo-transient iteration of
 * Alkhimenkov et al. (arXiv:2305.01701):
 *   - governing equations: Eqs. A22S, A21S, A23S (Sec. 2.5);
 *   - pseudo-transient form: Eqs. A22P, A2ssP, A23ssP (Sec. 3.2) with the
 *     numerical parameters of Eqs. PT1-PT24qq;
 *   - Jaumann rotation of the old stress: Eqs. j1-j14 and Appendix A;
 *   - Drucker-Prager yield and return: Eqs. A6-A6121lambda, Sec. 3.3;
 *   - pure-shear velocity walls with free slip: Eqs. A7-A9M (Sec. 4.1);
 *   - L-infinity convergence measures: Eqs. Convergence1-3 (Sec. 4.2).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an ep_status; on failure ep_last_error() holds a
 *     one-line reason.  A handle stays valid after EP_ERR_NOT_CONVERGED and
 *     keeps its last iterate.
 *   - Host arrays passed in are owned by the caller and copied before the
 *     call returns.  Device memory is owned by the library, or lives in a
 *     caller-provided workspace (see ep_create_grid).
 *   - Field arrays are FP64, compact, x fastest, in the natural extent of
 *     their staggered location: centres nx*ny[*nz]; x-faces (nx+1)*ny[*nz];
 *     y-faces nx*(ny+1)[*nz]; z-faces nx*ny*(nz+1); 2D vertices and 3D
 *     xy-edges (nx+1)*(ny+1)[*nz]; xz-edges (nx+1)*ny*(nz+1); yz-edges
 *     nx*(ny+1)*(nz+1).  The box is [-Lx/2, Lx/2] x [-Ly/2, Ly/2] [x ...].
 *   - Calls on one handle are not thread-safe; different handles are
 *     independent.  All device work of a handle runs on its stream.
 *   - No entry point launches work on a device other than the current one.
 */
#ifndef EP_H
#define EP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ep_grid *ep_handle;

typedef enum {
  EP_OK = 0,
  EP_ERR_ARG = 1,            /* invalid argument (sizes, psi != 0, nulls)   */
  EP_ERR_CUDA = 2,           /* a CUDA runtime call failed                  */
  EP_ERR_OOM = 3,            /* device allocation failed / workspace short  */
  EP_ERR_STATE = 4,          /* call out of order (e.g. solve w/o increment)*/
  EP_ERR_NOT_CONVERGED = 5,  /* max_iter reached; state kept                */
  EP_ERR_DIVERGED = 6,       /* NaN/Inf in a residual norm                  */
  EP_ERR_TIMEOUT = 7,        /* a bounded device wait gave up               */
  EP_PENDING = 8             /* ep_solve_chunks: not decided yet, continue  */
} ep_status;

/* EP_FP64: every sweep in FP64.  EP_FP32_MIXED: sweeps in FP32 on the
 * velocity increment of the current load increment, with FP64 residual
 * norms, convergence test, start-of-increment base state and history. */
typedef enum { EP_FP64 = 0, EP_FP32_MIXED = 1 } ep_precision;

/* pure-shear loading planes (Eqs. A7-A9M): XY is v_x = a x, v_y = -a y
 * (v_z = 0 in 3D); XZ is v_x = a x, v_z = -a z, v_y = 0 (3D only). */
enum { EP_LOAD_XY = 0, EP_LOAD_XZ = 1 };

/* field ids for ep_get_fields / ep_set_fields (FP64, layout above) */
enum {
  EP_VX = 0, EP_VY, EP_VZ,           /* converged velocity (faces)          */
  EP_TXX, EP_TYY, EP_TZZ,            /* deviatoric stress, centres          */
  EP_TXY, EP_TXZ, EP_TYZ,            /* deviatoric stress, vertices/edges   */
  EP_P,                              /* pressure, centres                   */
  EP_EPL,                            /* accumulated plastic strain, centres */
  EP_UX, EP_UY, EP_UZ,               /* displacement (faces)                */
  EP_EXX, EP_EYY, EP_EZZ,            /* accumulated total strain, centres   */
  EP_EXY, EP_EXZ, EP_EYZ,            /* accumulated total strain, edges     */
  EP_COH,                            /* cohesion, centres                   */
  EP_EII,                            /* sqrt(eps:eps/2) of EXX..EYZ (read)  */
  EP_SCALE,                          /* last return scale s, centres (read) */
  EP_V0X, EP_V0Y, EP_V0Z,            /* start velocity of the increment     */
  EP_FIELD_COUNT_ = 29
};

typedef struct {
  double tol;           /* stop when eps_res <= tol                           */
  long long max_iter;   /* iteration cap; a multiple of n_chk                 */
  int n_chk;            /* residual check cadence (even, >= 2)                */
  double c_cfl;         /* Vp = c_cfl * dx_min per pseudo step (0.9/sqrt(nd)) */
  double xi;            /* multiplier of Re_opt = 3 sqrt(10) pi / 2 (1)       */
  double r_pt;          /* K~/G~ of Eq. PT23 (r_opt = 1/2)                    */
  int jaumann;          /* rotate the old stress (Eq. j1), default 1          */
  /* frozen plasticity (Sec. 3.3): at the first check with k >= freeze_iter
   * and eps_rel > freeze_eps, the centre return scales are held for the rest
   * of the increment (the iteration becomes linear).  freeze_iter < 0 (the
   * default) follows the paper: 16 n_x for grids of more than 10^6 cells,
   * never otherwise; 0 never freezes. */
  long long freeze_iter;
  double freeze_eps;    /* default 1e-4                                        */
  /* advection of the old stress, the v_k d sigma_ij / dx_k term of the
   * Jaumann rate (Eq. j1; Fig. 1's adv kernels): when 1, every increment
   * after a committed one first transports tau_hat and p_hat over its dt with
   * the last converged velocity (explicit first-order upwind; zero gradient
   * at inflow walls; free-slip wall shear stays zero).  Stable for
   * max|v| dt / dx_min <= 1 / ndim.  The count of committed increments
   * decides: a grid resumed through ep_set_fields advects from its first
   * commit on, and ep_restore brings back the state before the advection of
   * the checkpointed increment.  Default 0 (off). */
  int advection;
  /* incompressible variant (Sec. 3.2, Eq. A2ssP2 in place of Eq. A2ssP):
   * the pressure is pseudo-time state stepped by -K~ div v (pseudo step 1),
   * starts at the old pressure, and its stopping measure is 2 eta_ve times
   * the interval-averaged |div v| relative to max|sigma|.  Default 0. */
  int incompressible;
  /* bound, in SM clock cycles, of each wait of the TMA sweep kernel
   * (EP_KERNEL_FUSED_TMA) for its plane copies; 0 (default) is 2^31 cycles,
   * about a second.  A wait that runs out ends the solve with
   * EP_ERR_TIMEOUT after the block has waited (with the default bound) for
   * the copies it issued; the handle stays usable. */
  long long wait_cycles;
} ep_solver_opts;

typedef struct {
  long long iters;      /* iteration index of the converged check            */
  double eps_res;       /* max(eps_mom, eps_tau, eps_p)                       */
  double eps_mom;       /* dx_min max|R| / max|sigma|         (Eq. Conv.3)    */
  double eps_tau;       /* max|d tau| / (1 - beta_tau) / max|sigma|           */
  double eps_p;         /* max|d p| / (1 - beta_p) / max|sigma|               */
  double eps_rel;       /* max|V - V_it| / max|V| between checks (Eq. Conv.2) */
  double max_r;         /* max|R| over interior faces                         */
  double max_sigma;     /* max|sigma_ij| over all components                  */
  long long n_plastic;  /* centres with s < 1 at convergence                  */
  double sxx_int_centre;/* integral of sigma_xx along the centre column       */
  double sxx_int_right; /* the same along the rightmost column                */
  double ms;            /* device wall time of the solve, milliseconds       */
  int status;           /* ep_status of the solve                             */
  long long frozen_at;  /* iteration at which the scales froze, -1 if never   */
} ep_solve_info;

/* Device bytes a grid needs.  Pass a buffer of at least this size to
 * ep_create_grid to keep every device allocation in caller memory. */
ep_status ep_workspace_bytes(int ndim, const int n[3], ep_precision prec, size_t *bytes);

/* Create a grid of n[0] x n[1] (x n[2]) cells on a box of size L (Sec. 3.1).
 * stream: a cudaStream_t or NULL (the library creates its own).
 * workspace: NULL (the library allocates with cudaMalloc) or a device
 * pointer of at least ep_workspace_bytes bytes, 256-byte aligned, owned by the
 * caller and kept alive until ep_destroy.  ndim must be 2 or 3, n >= 1. */
ep_status ep_create_grid(int ndim, const int n[3], const double L[3], ep_precision prec,
                         void *stream, void *workspace, size_t workspace_bytes, ep_handle *out);

/* Material (Sec. 2.2, Eqs. A43, A61, A611): bulk K and shear G moduli, shear
 * viscosity mu_s (INFINITY = elastic limit), friction angle phi and dilation
 * angle psi in degrees (psi must be 0, Eq. A6121lambda), and the per-cell
 * cohesion (host, nx*ny[*nz] values, copied; a value that is not finite
 * is rejected with EP_ERR_ARG). */
ep_status ep_set_material(ep_handle h, double K, double G, double mu_s, double phi_deg,
                          double psi_deg, const double *cohesion);

/* Per-cell shear modulus (the paper's heterogeneous G-bar of Sec. 4.1):
 * G (host, nx*ny[*nz] values > 0, copied) replaces the uniform G of
 * ep_set_material in the Maxwell law (Eqs. A43, A23ssP) point by point:
 * eta_ve and the weight c2 = eta_ve / (G dt) of the rotated old stress follow
 * G at the centres, and at a vertex/edge the mean G of the centres around it
 * (indices clamped at the walls); the pseudo-transient parameters (Eqs.
 * PT1-PT24qq) use the largest G.  NULL restores the uniform G.  Grids with a
 * per-cell G run the staged sweep kernels.  Not inside an open increment. */
ep_status ep_set_shear_modulus(ep_handle h, const double *G);

/* Fill opts with the defaults for a grid of dimension ndim. */
ep_status ep_default_solver(int ndim, ep_solver_opts *opts);
ep_status ep_set_solver(ep_handle h, const ep_solver_opts *opts);

/* Start a load increment of length dt with pure shear at rate a in
 * load_plane (Eqs. A7-A9M).  body_force: NULL or host face arrays
 * concatenated x, y[, z] (Eq. A220).  use_warm_start: non-zero adds the
 * attached warm-start predictor's velocity increment to the start. */
ep_status ep_apply_increment(ep_handle h, double a, double dt, int load_plane,
                             const double *body_force, int use_warm_start);

/* The same with an arbitrary diagonal velocity gradient rates[0..2] and an
 * optional host start increment dv_start (face arrays concatenated, walls
 * ignored) added to the previous converged velocity. */
ep_status ep_apply_increment_rates(ep_handle h, const double rates[3], double dt,
                                   const double *body_force, const double *dv_start);

/* Iterate the current increment to eps_res <= tol (or max_iter) and, on
 * success, commit the history (the "old" fields of Fig. 1).  info may be
 * NULL.  Returns EP_ERR_NOT_CONVERGED / EP_ERR_DIVERGED without committing. */
ep_status ep_solve_increment(ep_handle h, ep_solve_info *info);

/* Iterate the open increment for at most max_chunks chunks of n_chk
 * iterations (Sec. 3.2, the pseudo-time loop of Fig. 1, cut into pieces).
 * Returns EP_PENDING when the stopping test has not decided yet: the iterate,
 * the convergence record and the frozen-plasticity state are kept and the
 * next call continues the same iteration (info->iters is then the next check
 * iteration, info->ms the device time of this call).  Otherwise it returns
 * what ep_solve_increment returns and commits on convergence.  Calling it
 * until the status is not EP_PENDING performs exactly the iterations of one
 * ep_solve_increment; applying a new increment abandons an undecided solve. */
ep_status ep_solve_chunks(ep_handle h, int max_chunks, ep_solve_info *info);

/* Commit the current iterate as the increment's result (used after a
 * deliberate fixed-iteration solve). */
ep_status ep_commit_increment(ep_handle h);

/* Copy one FP64 field to/from host memory; count must equal the field's
 * size (ep_field_count).  ep_set_fields accepts history fields only. */
ep_status ep_field_count(ep_handle h, int field, size_t *count);
ep_status ep_get_fields(ep_handle h, int field, double *host_out, size_t count);
ep_status ep_set_fields(ep_handle h, int field, const double *host_in, size_t count);

/* Sweep kernel selection.  EP_KERNEL_AUTO (default): the fastest measured
 * kernel for the grid -- for FP32 grids the fused one-kernel sweep (2D) and
 * the register z-march sweep (3D), for FP64 grids the staged five-kernel
 * sweep (FP64 is bound by FP64 arithmetic on GB300, where the staged sweep
 * does no halo recomputation).
 * EP_KERNEL_STAGED / EP_KERNEL_FUSED force one;
 * EP_KERNEL_FUSED_TMA is the 3D fused sweep with every plane streamed by
 * the tensor-memory accelerator (a timed-out copy ends the solve with
 * EP_ERR_TIMEOUT); EP_KERNEL_FUSED_REG is the 3D fused sweep that keeps the
 * z-march in registers (lanes own x columns, warps own y rows).  The check
 * iteration of each chunk runs fused too with the FP32 register sweep (it
 * reduces the stopping measures itself); the other 3D flavours and FP64
 * grids take the staged sweep for it.  A body force always uses the staged
 * sweep.
 * shape (< 0 keeps the current): in 3D the z-planes per block of the fused
 * kernels (0, the default: chosen from the grid size so that the launch
 * fills every SM); in 2D the tile of the fused kernel (0: 32x8, 1: 32x16,
 * 2: 64x8 cells in shared memory; 3, 4: one warp per strip of 28 columns
 * marching 64 / 32 rows with its row history in registers). */
enum { EP_KERNEL_AUTO = -1, EP_KERNEL_STAGED = 0, EP_KERNEL_FUSED = 1, EP_KERNEL_FUSED_TMA = 2, EP_KERNEL_FUSED_REG = 3 };
ep_status ep_set_kernel(ep_handle h, int variant, int shape);

/* Batched 2D solves: many grids of any sizes and materials advance through
 * one persistent kernel per iteration (each block strides over (grid, tile)
 * work items; grids that have converged drop out), captured with the
 * per-grid residual checks into one CUDA graph per chunk of n_chk
 * iterations.  The grids must be 2D, share a precision and n_chk, and stay
 * alive until ep_destroy_batch; the batch runs on the first grid's stream.
 * A grid solved in a batch performs the same arithmetic as when solved
 * alone with the fused 2D kernel. */
typedef struct ep_batch *ep_batch_handle;
ep_status ep_create_batch(const ep_handle *grids, int count, ep_batch_handle *out);
/* start an increment in every grid: pure shear at rate a[i] (host array of
 * count rates) over dt, in the x-y plane */
ep_status ep_batch_apply_increment(ep_batch_handle b, const double *a, double dt);
/* iterate every grid to its tolerance and commit those that converged;
 * infos (nullable) receives count records; returns EP_ERR_NOT_CONVERGED /
 * EP_ERR_DIVERGED if any grid did not converge (the others are committed) */
ep_status ep_batch_solve_increment(ep_batch_handle b, ep_solve_info *infos);
/* time `iters` sweeps of each tile shape on the open increments, keep the
 * fastest (written to *tile_out when non-null) and restart the increments */
ep_status ep_batch_autotune(ep_batch_handle b, int iters, int *tile_out);
ep_status ep_batch_set_tile(ep_batch_handle b, int tile);
/* time `iters` sweeps of the current tile over every grid of the open
 * increments (all grids active, no checks): *ms_per_sweep receives the mean
 * device time of one sweep; the increments then start again */
ep_status ep_batch_time_sweep(ep_batch_handle b, int iters, double *ms_per_sweep);
ep_status ep_destroy_batch(ep_batch_handle b);

/* Learned warm start.  A convolutional U-Net (hand-written CUDA forward,
 * backward and Adam kernels; BF16 weights, FP32 accumulation and master
 * weights) predicts an increment's velocity change from the previous ones.
 * Layers: `levels` encoder levels of two 3^D convolutions + ReLU with
 * base * 2^l channels and average pooling, a mirrored decoder with nearest
 * upsampling and skip concatenation, and a zero-initialised 1^D head.
 * Tensors are FP32 device arrays N x C x [Z x] Y x X (x fastest); spatial
 * sizes must be multiples of 2^(levels-1). */
typedef struct ep_net *ep_net_handle;
ep_status ep_net_create(int ndim, int in_ch, int out_ch, int base, int levels, unsigned long long seed,
                        void *stream, ep_net_handle *out);
ep_status ep_net_param_count(ep_net_handle n, long long *count);
ep_status ep_net_get_params(ep_net_handle n, float *host, long long count);
ep_status ep_net_set_params(ep_net_handle n, const float *host, long long count);
/* y (device, N x out_ch x ...) = net(x); size = {X, Y[, Z]} */
ep_status ep_net_forward(ep_net_handle n, const float *x, int N, const int size[3], float *y);
/* ep_net_forward without any allocation.  The paper has no counterpart: this
 * serves callers that must not allocate device memory while they run -- a
 * solver loop applying the warm start between increments on a device whose
 * memory its arena and the caller's allocator pool already hold (a new
 * cudaMalloc may fail there), and latency-bound loops (cudaMalloc/cudaFree
 * synchronise the whole device).  The activations live in one static device
 * array of EP_NET_STATIC_FLOATS floats (64 MiB) inside the library, shared by
 * every call on a device: shapes whose activations need more return
 * EP_ERR_ARG (use ep_net_forward), and calls whose kernels may overlap on the
 * GPU (different streams with no ordering between them) race on it.  Nothing
 * in it has to start at zero.  The first call on a device looks up the
 * array's address with that device current; make it before any stream
 * capture.  The array is part of the library image: every device context in
 * which the library is loaded holds its 64 MiB, whether or not this entry
 * point is called.  The looked-up address is kept for the life of the
 * process, so resetting the device (cudaDeviceReset) and then calling this
 * again is not supported.  Arguments, layout and stream are those of
 * ep_net_forward. */
#define EP_NET_STATIC_FLOATS (16LL * 1024 * 1024)
ep_status ep_net_forward_static(ep_net_handle n, const float *x, int N, const int size[3], float *y);
/* MSE loss mean(((net(x) - t)/scale)^2) (scale: ep_net_set_output_scale,
 * default 1) and its parameter gradient (host, nullable) */
ep_status ep_net_gradients(ep_net_handle n, const float *x, const float *t, int N, const int size[3],
                           double *loss, float *grad_host, long long count);
/* one Adam step (beta 0.9 / 0.999) on the MSE loss; loss (nullable, host) */
ep_status ep_net_train_step(ep_net_handle n, const float *x, const float *t, int N, const int size[3], float lr,
                            double *loss);
/* The network's output is `scale` times its head's (default 1), and the
 * training loss is taken in units of the scale: mean(((net(x) - t)/scale)^2).
 * With the scale set to the training targets' root mean square the head's
 * values, the loss and the gradients stay of order one whatever the targets'
 * magnitude (Adam's epsilon then stays negligible).  0 makes the output zero
 * and the loss the targets' mean square. */
ep_status ep_net_set_output_scale(ep_net_handle n, double scale);
ep_status ep_net_get_output_scale(ep_net_handle n, double *scale);
ep_status ep_net_destroy(ep_net_handle n);
const char *ep_net_last_error(ep_net_handle n);

/* The learned warm start (the method's extension (a); the paper's own
 * iteration, Sec. 3.2, starts every increment from the previous one).  The
 * network works on a grid of coarse cells, each the mean of coarsen^D fine
 * cells, padded with zeros to a multiple of 4 cells per side
 * (ep_warm_dims).  Tensors are FP32, channels x [Z x] Y x X, x fastest.
 * Input channels (EP_WARM_IN: 13 in 3D, 9 in 2D), at cell centres:
 *   the previous increment's velocity change (centre mean per component)
 *   over S_v; the old deviator, normal components and shear components
 *   averaged from the 4 surrounding vertices/edges, over the cell's cohesion
 *   c; the old pressure over c; 1 - s (the last return scale); c / max c;
 *   the accumulated plastic strain over S_e.
 * Output channels (EP_WARM_OUT: 9 in 3D, 5 in 2D): the increment's velocity
 *   change over S_v (nd), then the converged pseudo-time stress state minus
 *   the physical response of the converged velocity over S_t (normal
 *   components, then shear components averaged to the centre).
 * S_v = 0.1 |a| L_max, S_t = 2 G |a| dt, S_e = 10 |a| dt, |a| the largest
 * loading rate of the grid's increment.  With a network attached,
 * ep_apply_increment(..., use_warm_start = 1) starts the interior velocity at
 * v + S_v * (velocity channels interpolated linearly from the coarse centres
 * to the faces) and the pseudo-time stress state at the physical response of
 * that velocity plus S_t * (stress channels interpolated to centres and
 * interior vertices/edges).  A zero output reproduces the plain start; the
 * iteration still runs to the same tolerance.  With fewer than two committed
 * increments the plain start is used. */
#define EP_WARM_IN(nd) ((nd) == 3 ? 13 : 9)
#define EP_WARM_OUT(nd) ((nd) == 3 ? 9 : 5)
/* Padded coarse size {X, Y, Z} (Z = 1 in 2D) for coarsening factor coarsen. */
ep_status ep_warm_dims(ep_handle h, int coarsen, int dims[3]);
/* Attach a network with EP_WARM_IN(ndim) inputs and EP_WARM_OUT(ndim)
 * outputs, applied at coarsening factor coarsen (>= 1); NULL detaches.  The
 * network must outlive the attachment. */
ep_status ep_attach_warm_start(ep_handle h, ep_net_handle net, int coarsen);
/* Recording on (non-zero): every later commit also keeps the physical
 * response of the converged velocity (one FP32 box per stress component,
 * allocated here), which ep_warm_target needs. */
ep_status ep_warm_record(ep_handle h, int on);
/* The features of the next increment at coarsening coarsen (device,
 * EP_WARM_IN x padded size).  Needs two committed increments. */
ep_status ep_warm_features(ep_handle h, int coarsen, float *dev_out);
/* After a recorded solve: that increment's target (device, EP_WARM_OUT x
 * padded size). */
ep_status ep_warm_target(ep_handle h, int coarsen, float *dev_out);

/* Device-resident checkpoint of the FP64 history (velocity and the one
 * before it, deviator, pressure, plastic strain, displacement, accumulated
 * strain) and of the last return scale (a warm-start feature).  The first
 * ep_snapshot allocates the checkpoint with cudaMalloc (freed by ep_destroy);
 * ep_restore copies it back, so the next increment starts from the saved
 * state.  Both run on the grid's stream and return after it has drained. */
ep_status ep_snapshot(ep_handle h);
ep_status ep_restore(ep_handle h);

/* Profiling: run `iters` pseudo-time sweeps (no residual checks) from the
 * current state on the grid's stream, timing each kernel with CUDA events.
 * ms_out[0..n_out-1] receives the mean milliseconds per launch of each sweep
 * kernel in launch order, followed by the mean milliseconds of one whole
 * iteration; n_kernels (nullable) receives the number of sweep kernels.
 * The sweep state afterwards is unspecified: call it between increments. */
ep_status ep_time_sweep(ep_handle h, int iters, double *ms_out, int n_out, int *n_kernels);

/* Algorithmic bytes one sweep iteration must move per cell in the grid's
 * precision (the fused-sweep lower bound: every state array read and
 * written once, every constant read once). */
ep_status ep_sweep_bytes_per_cell(ep_handle h, double *bytes);

/* Measurement: the current device's FP64 fused multiply-add rate in
 * TFLOP/s (2 flops per FMA; independent register chains, no memory traffic,
 * best of five launches timed with CUDA events).  The FP64 sweeps are bound
 * by FP64 arithmetic on GB300, so this is the roof they are reported
 * against. */
ep_status ep_measure_fp64_peak(double *tflops);

ep_status ep_destroy(ep_handle h);

/* Last error message of h, or of the calling thread when h is NULL. */
const char *ep_last_error(ep_handle h);

#ifdef __cplusplus
}
#endif
#endif /* EP_H */
