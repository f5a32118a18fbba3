/*
 * ep_oracle.c -- plain, slow FP64 CPU oracle of the pseudo-transient
 * elasto-plastic staggered-grid solve (Alkhimenkov et al., arXiv:2305.01701).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path never
 * calls it and shares no code with it: the only thing both sides take from a
 * common place is the seeded input arrays.
 *
 * Every step is written out in the order the paper states it, one plain loop
 * per quantity, with no fusion or reordering:
 *   strain rate and spin ............ Eq. A41 (strain rate), Eq. A5 (vorticity)
 *   rotated (Jaumann) history ....... Eqs. j1-j14 and Appendix A
 *   pseudo-transient pressure ....... Eq. A2ssP
 *   pseudo-transient deviator ....... Eq. A23ssP (Maxwell, Eq. A43)
 *   Drucker-Prager return ........... Eqs. A6, A61, A611, A6121lambda; Sec. 3.3
 *   stress divergence ............... Eq. A22S with body force (Eq. A220)
 *   pseudo-transient momentum ....... Eq. A22P
 *   numerical parameters ............ Eqs. PT1-PT24qq
 *   L-infinity convergence norms .... Eqs. Convergence1-3
 *   history commit .................. the "old" fields of Fig. 1
 *
 * Readings where the paper is silent or garbled:
 *  - J2 squares its shear terms (the printed 2D/3D formulas drop the squares);
 *  - 2D carries no tau_zz and uses J2 = (txx^2 + tyy^2)/2 + txy^2;
 *  - spin w_xy = (dvx/dy - dvy/dx)/2, the textbook Jaumann sign;
 *  - centred box [-L/2, L/2]; free slip = zero shear stress, shear strain rate
 *    and spin on wall vertices/edges, prescribed normal velocity on walls;
 *  - yield is evaluated at cell centres with shear components averaged from
 *    the 4 surrounding vertices/edges; a vertex/edge takes the arithmetic mean
 *    of the scale factors of its 4 adjacent centres;
 *  - the return scales the relaxed trial deviator by s = Y / sqrt(J2), with
 *    Y = max(0, A p + B c), when sqrt(J2) > Y;
 *  - the history is rotated with the current iterate's spin at every
 *    iteration (explicit in the old stress, implicit in the spin); products
 *    are formed where both factors live and averaged to the target location;
 *  - pseudo-time step 1, Vp = C dx_min, eta = eta_ve in Eq. PT1, L = L_max;
 *  - optional advection of the old stress (the v_k d sigma_ij / dx_k term of
 *    Eq. j1; the paper names its kernels adv1/adv2 in Fig. 1 but prints no
 *    discretisation): once per increment, explicit first-order upwind
 *    transport of the history deviator and pressure over dt with the
 *    previous increment's converged velocity (see advect_history);
 *  - optional incompressible variant (Eq. A2ssP2 in place of Eq. A2ssP): the
 *    pressure is pseudo-time state stepped by -K~ div v, starts at p_hat, and
 *    its stopping measure is 2 eta_ve times the interval-averaged divergence
 *    (see or_set_incompressible);
 *  - optional per-cell shear modulus (the paper's Gaussian G-bar, Sec. 4.1):
 *    eta_ve and the weight of the rotated old stress follow G point by point,
 *    a vertex/edge takes the arithmetic mean of its adjacent centres' G, and
 *    the pseudo-transient parameters use the largest G (see
 *    or_set_shear_modulus);
 *  - each iteration starts from the stress consistent with the start
 *    velocity (one pseudo step with no relaxation memory);
 *  - the stopping test takes the largest of the three equations' residuals,
 *    each in stress units and relative to max|sigma|, every n_chk iterations;
 *    each residual is the pseudo-time rate of its state (velocity, deviator,
 *    pressure) averaged over the check interval.
 *
 * Threads: the loops of one iteration that write one element per loop index
 * carry OpenMP pragmas; norms and reductions stay serial.  Each element's
 * arithmetic is the same on any thread, so a build with -fopenmp gives the
 * same bits as the plain build (the default, which ignores the pragmas).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- status codes and field ids (same numbering as the library's API) ---- */
enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_OOM = 3, OR_ERR_STATE = 4,
       OR_ERR_NOT_CONVERGED = 5, OR_ERR_DIVERGED = 6 };

enum {
  OF_VX = 0, OF_VY, OF_VZ,
  OF_TXX, OF_TYY, OF_TZZ, OF_TXY, OF_TXZ, OF_TYZ,
  OF_P, OF_EPL,
  OF_UX, OF_UY, OF_UZ,
  OF_EXX, OF_EYY, OF_EZZ, OF_EXY, OF_EXZ, OF_EYZ,
  OF_COH, OF_EII, OF_SCALE,
  OF_V0X, OF_V0Y, OF_V0Z,
  OF_RX, OF_RY, OF_RZ,
  OF_COUNT
};

typedef struct {
  long iters;
  double eps_res, eps_mom, eps_tau, eps_p, eps_rel, max_r, max_sigma;
  long n_plastic;
  double sxx_int_centre, sxx_int_right;
  int status;
  long frozen_at;   /* iteration at which the return scales were frozen, -1 if never */
} or_info;

typedef struct {
  int ndim, nx, ny, nz;
  double L[3], dx, dy, dz;
  /* material (Eqs. A43, A61, A611, A6121) */
  double K, G, mu_s, A, B;
  double *coh;
  double *Gc;     /* per-centre shear modulus (NULL: the uniform G) */
  double Gref;    /* its largest value, for the pseudo-transient parameters */
  int have_material;
  /* solver settings */
  double tol, c_cfl, xi, r_pt;
  long max_iter;
  int n_chk, jaumann;
  /* frozen plasticity (Sec. 3.3): from the first check at k >= freeze_iter
   * with eps_rel > freeze_eps on, the centre scales s keep their values */
  long freeze_iter;   /* 0: never */
  double freeze_eps;
  int frozen;
  /* advection of the old stress (Eq. j1), once per committed increment */
  int advect;
  /* incompressible pressure equation (Eq. A2ssP2) instead of Eq. A2ssP */
  int incompressible;
  long commits, adv_done;
  /* loading of the current increment (Eqs. A7-A9M) */
  double rate[3], dt;
  double *f[3];
  int started, in_increment, evaluated;
  /* history (the "old" fields: hat quantities of Eqs. A2ssP, A23ssP) */
  double *v[3];
  double *tn[3], *ts[3];
  double *p;
  double *epl;
  double *u[3];
  double *an[3], *as[3];
  /* pseudo-time state: velocity, deviator, pressure */
  double *v0[3], *vi[3], *vchk[3];
  double *tn_k[3], *ts_k[3], *p_k;
  double *tn_c[3], *ts_c[3], *p_c;   /* stress state at the previous check */
  /* quantities of the last evaluation */
  double *en[3], *es[3], *om[3], *div;
  double *tJn[3], *tJs[3];
  double *trn[3], *trs[3];
  double *Tn[3], *Ts[3];
  double *pc, *s;
  double *sn[3], *ss[3];
  double *R[3];
} or_grid;

/* ------------------------------------------------------------------------ */
/* sizes of each staggered location                                          */
/* ------------------------------------------------------------------------ */
static long n_centres(const or_grid *g) { return (long)g->nx * g->ny * g->nz; }

static void face_dims(const or_grid *g, int d, int *ex, int *ey, int *ez) {
  *ex = g->nx + (d == 0); *ey = g->ny + (d == 1); *ez = g->nz + (d == 2 && g->ndim == 3);
}
static long n_face(const or_grid *g, int d) {
  int ex, ey, ez; face_dims(g, d, &ex, &ey, &ez); return (long)ex * ey * ez;
}
/* shear location c: 0 = xy (2D vertices / 3D xy-edges), 1 = xz, 2 = yz */
static void shear_dims(const or_grid *g, int c, int *ex, int *ey, int *ez) {
  if (g->ndim == 2) { *ex = g->nx + 1; *ey = g->ny + 1; *ez = 1; return; }
  *ex = g->nx + (c != 2); *ey = g->ny + (c != 1); *ez = g->nz + (c != 0);
}
static long n_shear(const or_grid *g, int c) {
  int ex, ey, ez; shear_dims(g, c, &ex, &ey, &ez); return (long)ex * ey * ez;
}
static int n_shear_comp(const or_grid *g) { return g->ndim == 3 ? 3 : 1; }

/* index helpers, x fastest */
#define CI(i, j, k)  (((long)(k) * g->ny + (j)) * g->nx + (i))
#define FXI(i, j, k) (((long)(k) * g->ny + (j)) * (g->nx + 1) + (i))
#define FYI(i, j, k) (((long)(k) * (g->ny + 1) + (j)) * g->nx + (i))
#define FZI(i, j, k) (((long)(k) * g->ny + (j)) * g->nx + (i))
#define XYI(i, j, k) (((long)(k) * (g->ny + 1) + (j)) * (g->nx + 1) + (i))
#define XZI(i, j, k) (((long)(k) * g->ny + (j)) * (g->nx + 1) + (i))
#define YZI(i, j, k) (((long)(k) * (g->ny + 1) + (j)) * g->nx + (i))

static double *zalloc(long n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

void or_destroy(or_grid *g);

or_grid *or_create(int ndim, const int *n, const double *L) {
  if (ndim != 2 && ndim != 3) return NULL;
  for (int d = 0; d < ndim; ++d) if (n[d] < 1 || !(L[d] > 0.0)) return NULL;
  or_grid *g = (or_grid *)calloc(1, sizeof(or_grid));
  g->ndim = ndim; g->nx = n[0]; g->ny = n[1]; g->nz = ndim == 3 ? n[2] : 1;
  g->L[0] = L[0]; g->L[1] = L[1]; g->L[2] = ndim == 3 ? L[2] : 1.0;
  g->dx = g->L[0] / g->nx; g->dy = g->L[1] / g->ny; g->dz = g->L[2] / g->nz;
  g->tol = 1e-8; g->max_iter = 1000000; g->n_chk = 100;
  g->freeze_iter = 0; g->freeze_eps = 1e-4; g->frozen = 0;
  g->c_cfl = 0.9 / sqrt((double)ndim); g->xi = 1.0; g->r_pt = 0.5; g->jaumann = 1;
  long nc = n_centres(g);
  g->coh = zalloc(nc); g->p = zalloc(nc); g->epl = zalloc(nc); g->div = zalloc(nc);
  g->pc = zalloc(nc); g->s = zalloc(nc); g->p_k = zalloc(nc); g->p_c = zalloc(nc);
  for (int d = 0; d < 3; ++d) {
    long nf = d < ndim ? n_face(g, d) : 0;
    g->v[d] = zalloc(nf); g->u[d] = zalloc(nf); g->v0[d] = zalloc(nf); g->vi[d] = zalloc(nf);
    g->vchk[d] = zalloc(nf); g->R[d] = zalloc(nf); g->f[d] = zalloc(nf);
    long nn = d < ndim ? nc : 0;
    g->tn[d] = zalloc(nn); g->an[d] = zalloc(nn); g->en[d] = zalloc(nn); g->tn_k[d] = zalloc(nn);
    g->tJn[d] = zalloc(nn); g->trn[d] = zalloc(nn); g->Tn[d] = zalloc(nn); g->sn[d] = zalloc(nn);
    g->tn_c[d] = zalloc(nn);
    long ns = (ndim == 3 || d == 0) ? n_shear(g, d) : 0;
    g->ts[d] = zalloc(ns); g->as[d] = zalloc(ns); g->es[d] = zalloc(ns); g->om[d] = zalloc(ns);
    g->ts_k[d] = zalloc(ns); g->tJs[d] = zalloc(ns); g->trs[d] = zalloc(ns); g->Ts[d] = zalloc(ns);
    g->ss[d] = zalloc(ns); g->ts_c[d] = zalloc(ns);
  }
  return g;
}

void or_destroy(or_grid *g) {
  if (!g) return;
  free(g->Gc);
  free(g->coh); free(g->p); free(g->epl); free(g->div); free(g->pc); free(g->s); free(g->p_k); free(g->p_c);
  for (int d = 0; d < 3; ++d) {
    free(g->v[d]); free(g->u[d]); free(g->v0[d]); free(g->vi[d]); free(g->vchk[d]);
    free(g->R[d]); free(g->f[d]);
    free(g->tn[d]); free(g->an[d]); free(g->en[d]); free(g->tn_k[d]); free(g->tJn[d]);
    free(g->trn[d]); free(g->Tn[d]); free(g->sn[d]);
    free(g->ts[d]); free(g->as[d]); free(g->es[d]); free(g->om[d]); free(g->ts_k[d]);
    free(g->tJs[d]); free(g->trs[d]); free(g->Ts[d]); free(g->ss[d]);
    free(g->tn_c[d]); free(g->ts_c[d]);
  }
  free(g);
}

/* Material: K, G, shear viscosity mu_s (INFINITY = elastic limit), friction
 * angle phi and dilation angle psi (must be 0: the return of Eq. A6121lambda
 * assumes psi = 0).  A, B follow Eq. A61 in 2D and Eqs. A611 in 3D. */
int or_set_material(or_grid *g, double K, double G, double mu_s, double phi_deg,
                    double psi_deg, const double *coh) {
  if (!(K > 0.0) || !(G > 0.0) || !(mu_s > 0.0) || psi_deg != 0.0) return OR_ERR_ARG;
  const double phi = phi_deg * M_PI / 180.0;
  g->K = K; g->G = G; g->mu_s = mu_s;
  if (g->ndim == 2) {
    g->A = sin(phi); g->B = cos(phi);
  } else {
    g->A = 6.0 * sin(phi) / (sqrt(3.0) * (3.0 - sin(phi)));
    g->B = 6.0 * cos(phi) / (sqrt(3.0) * (3.0 - sin(phi)));
  }
  memcpy(g->coh, coh, sizeof(double) * n_centres(g));
  g->have_material = 1;
  return OR_OK;
}

int or_set_solver(or_grid *g, double tol, long max_iter, int n_chk, double c_cfl, double xi,
                  double r_pt, int jaumann) {
  if (!(tol >= 0.0) || max_iter < 0 || n_chk < 1 || !(c_cfl > 0.0) || !(xi > 0.0) || !(r_pt > 0.0))
    return OR_ERR_ARG;
  g->tol = tol; g->max_iter = max_iter; g->n_chk = n_chk; g->c_cfl = c_cfl; g->xi = xi; g->r_pt = r_pt;
  g->jaumann = jaumann != 0;
  return OR_OK;
}

/* Frozen plasticity (Sec. 3.3, last paragraph): the paper stops updating the
 * plastic multiplier when an increment still has eps_rel > 1e-4 after
 * 16 n_x iterations and iterates the then-linear problem to tolerance.  Here:
 * at the first check with k >= freeze_iter and eps_rel > freeze_eps, the
 * centre scales s of that iteration are kept for the rest of the increment
 * (edges keep using the mean of their adjacent centre scales).  freeze_iter
 * = 0 never freezes. */
int or_set_freeze(or_grid *g, long freeze_iter, double freeze_eps) {
  if (freeze_iter < 0 || !(freeze_eps >= 0.0)) return OR_ERR_ARG;
  g->freeze_iter = freeze_iter;
  g->freeze_eps = freeze_eps;
  return OR_OK;
}

static double spacing(const or_grid *g, int d) { return d == 0 ? g->dx : d == 1 ? g->dy : g->dz; }
static int is_boundary_face(const or_grid *g, int d, int i, int j, int k) {
  return d == 0 ? (i == 0 || i == g->nx) : d == 1 ? (j == 0 || j == g->ny) : (k == 0 || k == g->nz);
}

/* viscoelastic effective viscosity eta_ve = (1/(G dt) + 1/mu_s)^-1, the
 * coefficient of Eq. A23ssP at pseudo-steady state; mu_s = inf gives G dt. */
static double eta_for(const or_grid *g, double G) {
  return isinf(g->mu_s) ? G * g->dt : 1.0 / (1.0 / (G * g->dt) + 1.0 / g->mu_s);
}
/* the viscosity the pseudo-transient parameters use (the largest G) */
static double eta_ve(const or_grid *g) { return eta_for(g, g->Gc ? g->Gref : g->G); }
/* shear modulus at a centre */
static double G_centre(const or_grid *g, long c) { return g->Gc ? g->Gc[c] : g->G; }
/* shear modulus at point (i, j, k) of shear component s (2D vertices, 3D
 * edges): the mean over the centres around it (one layer in each dimension
 * where the point sits at cell centres, two where it sits on grid lines;
 * indices clamped at the walls, whose shear stress is zero anyway) */
static double G_shear(const or_grid *g, int s, int i, int j, int k) {
  if (!g->Gc) return g->G;
  const int st[3] = {g->ndim == 2 ? 1 : s != 2, g->ndim == 2 ? 1 : s != 1, g->ndim == 2 ? 0 : s != 0};
  const int q[3] = {i, j, k}, n[3] = {g->nx, g->ny, g->nz};
  double sum = 0.0;
  int cnt = 0;
  for (int c = -st[2]; c <= 0; ++c)
    for (int b = -st[1]; b <= 0; ++b)
      for (int a = -st[0]; a <= 0; ++a) {
        int idx[3] = {q[0] + a, q[1] + b, q[2] + c};
        for (int d = 0; d < 3; ++d) idx[d] = idx[d] < 0 ? 0 : idx[d] > n[d] - 1 ? n[d] - 1 : idx[d];
        sum += g->Gc[CI(idx[0], idx[1], idx[2])];
        ++cnt;
      }
  return sum / cnt;
}

/* ------------------------------------------------------------------------ */
/* Step 1: strain rates and spins (Eqs. A41, A5)                             */
/* ------------------------------------------------------------------------ */
static void strain_rates(or_grid *g, double *const vv[3]) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  const double dx = g->dx, dy = g->dy, dz = g->dz;
  double *vx = vv[0], *vy = vv[1], *vz = vv[2];
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
    long c = CI(i, j, k);
    g->en[0][c] = (vx[FXI(i + 1, j, k)] - vx[FXI(i, j, k)]) / dx;
    g->en[1][c] = (vy[FYI(i, j + 1, k)] - vy[FYI(i, j, k)]) / dy;
    g->div[c] = g->en[0][c] + g->en[1][c];
    if (g->ndim == 3) {
      g->en[2][c] = (vz[FZI(i, j, k + 1)] - vz[FZI(i, j, k)]) / dz;
      g->div[c] += g->en[2][c];
    }
  }
  /* xy: 2D vertices or 3D xy-edges; walls carry zero */
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k) for (int j = 0; j <= ny; ++j) for (int i = 0; i <= nx; ++i) {
    long e = XYI(i, j, k);
    if (i == 0 || i == nx || j == 0 || j == ny) { g->es[0][e] = 0.0; g->om[0][e] = 0.0; continue; }
    double a = (vx[FXI(i, j, k)] - vx[FXI(i, j - 1, k)]) / dy;   /* dvx/dy */
    double b = (vy[FYI(i, j, k)] - vy[FYI(i - 1, j, k)]) / dx;   /* dvy/dx */
    g->es[0][e] = 0.5 * (a + b);
    g->om[0][e] = 0.5 * (a - b);
  }
  if (g->ndim == 2) return;
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k <= nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i <= nx; ++i) {
    long e = XZI(i, j, k);
    if (i == 0 || i == nx || k == 0 || k == nz) { g->es[1][e] = 0.0; g->om[1][e] = 0.0; continue; }
    double a = (vx[FXI(i, j, k)] - vx[FXI(i, j, k - 1)]) / dz;   /* dvx/dz */
    double b = (vz[FZI(i, j, k)] - vz[FZI(i - 1, j, k)]) / dx;   /* dvz/dx */
    g->es[1][e] = 0.5 * (a + b);
    g->om[1][e] = 0.5 * (a - b);
  }
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k <= nz; ++k) for (int j = 0; j <= ny; ++j) for (int i = 0; i < nx; ++i) {
    long e = YZI(i, j, k);
    if (j == 0 || j == ny || k == 0 || k == nz) { g->es[2][e] = 0.0; g->om[2][e] = 0.0; continue; }
    double a = (vy[FYI(i, j, k)] - vy[FYI(i, j, k - 1)]) / dz;   /* dvy/dz */
    double b = (vz[FZI(i, j, k)] - vz[FZI(i, j - 1, k)]) / dy;   /* dvz/dy */
    g->es[2][e] = 0.5 * (a + b);
    g->om[2][e] = 0.5 * (a - b);
  }
}

/* ------------------------------------------------------------------------ */
/* Step 2: rotated history tau_J = tau_hat + dt * tau_R (Eq. j14, App. A)    */
/* ------------------------------------------------------------------------ */
static void rotated_history_2d(or_grid *g) {
  const int nx = g->nx, ny = g->ny;
  const double dt = g->dt;
  double *txy = g->ts[0], *wxy = g->om[0];
  #pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
    long c = CI(i, j, 0);
    double q = 0.0;
    if (g->jaumann)
      q = 0.25 * (txy[XYI(i, j, 0)] * wxy[XYI(i, j, 0)] + txy[XYI(i + 1, j, 0)] * wxy[XYI(i + 1, j, 0)] +
                  txy[XYI(i, j + 1, 0)] * wxy[XYI(i, j + 1, 0)] + txy[XYI(i + 1, j + 1, 0)] * wxy[XYI(i + 1, j + 1, 0)]);
    g->tJn[0][c] = g->tn[0][c] + dt * (2.0 * q);    /* R_xx =  2 t_xy w_xy */
    g->tJn[1][c] = g->tn[1][c] + dt * (-2.0 * q);   /* R_yy = -2 t_xy w_xy */
  }
  #pragma omp parallel for schedule(static)
  for (int j = 0; j <= ny; ++j) for (int i = 0; i <= nx; ++i) {
    long e = XYI(i, j, 0);
    if (i == 0 || i == nx || j == 0 || j == ny) { g->tJs[0][e] = 0.0; continue; }
    double r = 0.0;
    if (g->jaumann) {
      double dyx = 0.25 * ((g->tn[1][CI(i - 1, j - 1, 0)] - g->tn[0][CI(i - 1, j - 1, 0)]) +
                           (g->tn[1][CI(i, j - 1, 0)] - g->tn[0][CI(i, j - 1, 0)]) +
                           (g->tn[1][CI(i - 1, j, 0)] - g->tn[0][CI(i - 1, j, 0)]) +
                           (g->tn[1][CI(i, j, 0)] - g->tn[0][CI(i, j, 0)]));
      r = wxy[e] * dyx;                              /* R_xy = w_xy (t_yy - t_xx) */
    }
    g->tJs[0][e] = txy[e] + dt * r;
  }
}

static void rotated_history_3d(or_grid *g) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  const double dt = g->dt;
  double *txy = g->ts[0], *txz = g->ts[1], *tyz = g->ts[2];
  double *wxy = g->om[0], *wxz = g->om[1], *wyz = g->om[2];
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
    long c = CI(i, j, k);
    double pxy = 0.0, pxz = 0.0, pyz = 0.0;
    if (g->jaumann) {
      pxy = 0.25 * (txy[XYI(i, j, k)] * wxy[XYI(i, j, k)] + txy[XYI(i + 1, j, k)] * wxy[XYI(i + 1, j, k)] +
                    txy[XYI(i, j + 1, k)] * wxy[XYI(i, j + 1, k)] + txy[XYI(i + 1, j + 1, k)] * wxy[XYI(i + 1, j + 1, k)]);
      pxz = 0.25 * (txz[XZI(i, j, k)] * wxz[XZI(i, j, k)] + txz[XZI(i + 1, j, k)] * wxz[XZI(i + 1, j, k)] +
                    txz[XZI(i, j, k + 1)] * wxz[XZI(i, j, k + 1)] + txz[XZI(i + 1, j, k + 1)] * wxz[XZI(i + 1, j, k + 1)]);
      pyz = 0.25 * (tyz[YZI(i, j, k)] * wyz[YZI(i, j, k)] + tyz[YZI(i, j + 1, k)] * wyz[YZI(i, j + 1, k)] +
                    tyz[YZI(i, j, k + 1)] * wyz[YZI(i, j, k + 1)] + tyz[YZI(i, j + 1, k + 1)] * wyz[YZI(i, j + 1, k + 1)]);
    }
    g->tJn[0][c] = g->tn[0][c] + dt * (2.0 * (pxy + pxz));      /* R_xx */
    g->tJn[1][c] = g->tn[1][c] + dt * (-2.0 * (pxy - pyz));     /* R_yy */
    g->tJn[2][c] = g->tn[2][c] + dt * (-2.0 * (pxz + pyz));     /* R_zz */
  }
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k) for (int j = 0; j <= ny; ++j) for (int i = 0; i <= nx; ++i) {
    long e = XYI(i, j, k);
    if (i == 0 || i == nx || j == 0 || j == ny) { g->tJs[0][e] = 0.0; continue; }
    double r = 0.0;
    if (g->jaumann) {
      double dyx = 0.25 * ((g->tn[1][CI(i - 1, j - 1, k)] - g->tn[0][CI(i - 1, j - 1, k)]) +
                           (g->tn[1][CI(i, j - 1, k)] - g->tn[0][CI(i, j - 1, k)]) +
                           (g->tn[1][CI(i - 1, j, k)] - g->tn[0][CI(i - 1, j, k)]) +
                           (g->tn[1][CI(i, j, k)] - g->tn[0][CI(i, j, k)]));
      double Tyz = 0.25 * (tyz[YZI(i - 1, j, k)] + tyz[YZI(i, j, k)] + tyz[YZI(i - 1, j, k + 1)] + tyz[YZI(i, j, k + 1)]);
      double Wyz = 0.25 * (wyz[YZI(i - 1, j, k)] + wyz[YZI(i, j, k)] + wyz[YZI(i - 1, j, k + 1)] + wyz[YZI(i, j, k + 1)]);
      double Txz = 0.25 * (txz[XZI(i, j - 1, k)] + txz[XZI(i, j, k)] + txz[XZI(i, j - 1, k + 1)] + txz[XZI(i, j, k + 1)]);
      double Wxz = 0.25 * (wxz[XZI(i, j - 1, k)] + wxz[XZI(i, j, k)] + wxz[XZI(i, j - 1, k + 1)] + wxz[XZI(i, j, k + 1)]);
      r = wxy[e] * dyx + Tyz * Wxz + Txz * Wyz;   /* R_xy */
    }
    g->tJs[0][e] = txy[e] + dt * r;
  }
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k <= nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i <= nx; ++i) {
    long e = XZI(i, j, k);
    if (i == 0 || i == nx || k == 0 || k == nz) { g->tJs[1][e] = 0.0; continue; }
    double r = 0.0;
    if (g->jaumann) {
      double dzx = 0.25 * ((g->tn[2][CI(i - 1, j, k - 1)] - g->tn[0][CI(i - 1, j, k - 1)]) +
                           (g->tn[2][CI(i, j, k - 1)] - g->tn[0][CI(i, j, k - 1)]) +
                           (g->tn[2][CI(i - 1, j, k)] - g->tn[0][CI(i - 1, j, k)]) +
                           (g->tn[2][CI(i, j, k)] - g->tn[0][CI(i, j, k)]));
      double Tyz = 0.25 * (tyz[YZI(i - 1, j, k)] + tyz[YZI(i, j, k)] + tyz[YZI(i - 1, j + 1, k)] + tyz[YZI(i, j + 1, k)]);
      double Wyz = 0.25 * (wyz[YZI(i - 1, j, k)] + wyz[YZI(i, j, k)] + wyz[YZI(i - 1, j + 1, k)] + wyz[YZI(i, j + 1, k)]);
      double Txy = 0.25 * (txy[XYI(i, j, k - 1)] + txy[XYI(i, j + 1, k - 1)] + txy[XYI(i, j, k)] + txy[XYI(i, j + 1, k)]);
      double Wxy = 0.25 * (wxy[XYI(i, j, k - 1)] + wxy[XYI(i, j + 1, k - 1)] + wxy[XYI(i, j, k)] + wxy[XYI(i, j + 1, k)]);
      r = wxz[e] * dzx + Tyz * Wxy - Txy * Wyz;   /* R_xz */
    }
    g->tJs[1][e] = txz[e] + dt * r;
  }
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k <= nz; ++k) for (int j = 0; j <= ny; ++j) for (int i = 0; i < nx; ++i) {
    long e = YZI(i, j, k);
    if (j == 0 || j == ny || k == 0 || k == nz) { g->tJs[2][e] = 0.0; continue; }
    double r = 0.0;
    if (g->jaumann) {
      double dzy = 0.25 * ((g->tn[2][CI(i, j - 1, k - 1)] - g->tn[1][CI(i, j - 1, k - 1)]) +
                           (g->tn[2][CI(i, j, k - 1)] - g->tn[1][CI(i, j, k - 1)]) +
                           (g->tn[2][CI(i, j - 1, k)] - g->tn[1][CI(i, j - 1, k)]) +
                           (g->tn[2][CI(i, j, k)] - g->tn[1][CI(i, j, k)]));
      double Txy = 0.25 * (txy[XYI(i, j, k - 1)] + txy[XYI(i + 1, j, k - 1)] + txy[XYI(i, j, k)] + txy[XYI(i + 1, j, k)]);
      double Wxy = 0.25 * (wxy[XYI(i, j, k - 1)] + wxy[XYI(i + 1, j, k - 1)] + wxy[XYI(i, j, k)] + wxy[XYI(i + 1, j, k)]);
      double Txz = 0.25 * (txz[XZI(i, j - 1, k)] + txz[XZI(i + 1, j - 1, k)] + txz[XZI(i, j, k)] + txz[XZI(i + 1, j, k)]);
      double Wxz = 0.25 * (wxz[XZI(i, j - 1, k)] + wxz[XZI(i + 1, j - 1, k)] + wxz[XZI(i, j, k)] + wxz[XZI(i + 1, j, k)]);
      r = wyz[e] * dzy - Txy * Wxz - Txz * Wxy;   /* R_yz */
    }
    g->tJs[2][e] = tyz[e] + dt * r;
  }
}

/* ------------------------------------------------------------------------ */
/* Step 3: physical Maxwell trial deviator tau_tr = 2 eta_ve (eps_dev +      */
/* tau_J / (2 G dt)): the pseudo-steady solution of Eq. A23ssP without the   */
/* plastic term.  Walls carry zero.                                          */
/* ------------------------------------------------------------------------ */
static void trial(or_grid *g) {
  long nc = n_centres(g);
  #pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    const double G = G_centre(g, c), eta = eta_for(g, G), c2 = eta / (G * g->dt);
    for (int d = 0; d < g->ndim; ++d)
      g->trn[d][c] = 2.0 * eta * (g->en[d][c] - g->div[c] / 3.0) + c2 * g->tJn[d][c];
  }
  for (int s = 0; s < n_shear_comp(g); ++s) {
    int ex, ey, ez; shear_dims(g, s, &ex, &ey, &ez);
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < ez; ++k) for (int j = 0; j < ey; ++j) for (int i = 0; i < ex; ++i) {
      const long e = ((long)k * ey + j) * ex + i;
      const double G = G_shear(g, s, i, j, k), eta = eta_for(g, G), c2 = eta / (G * g->dt);
      g->trs[s][e] = 2.0 * eta * g->es[s][e] + c2 * g->tJs[s][e];
    }
  }
}

/* pseudo-transient parameters (Eqs. PT1-PT24qq) with pseudo-time step 1:
 * Vp = C dx_min, rho~ = Re eta_ve / (Vp L), G~ = rho~ Vp^2 / (r + 4/3),
 * K~ = r G~, Re = xi * 3 sqrt(10) pi / 2 and r = r_pt (Eqs. PT24q-PT24qq give
 * xi = 1 and r_pt = 1/2 for the incompressible viscous limit).  Returned as the relaxation
 * weights of Eqs. A2ssP/A23ssP after one implicit pseudo step,
 *   beta_tau = (1/(2 G~)) / (1/(2 G~) + 1/(2 eta_ve)),
 *   beta_p   = (1/K~) / (1/K~ + 1/(K dt)),
 * and the velocity step 1/rho~ of Eq. A22P. */
typedef struct { double beta_tau, beta_p, vstep, Gt, Kt, rho; } pt_t;

static double dx_min(const or_grid *g) {
  double m = g->dx < g->dy ? g->dx : g->dy;
  if (g->ndim == 3 && g->dz < m) m = g->dz;
  return m;
}

static pt_t pt_params(const or_grid *g) {
  pt_t q;
  double Lm = g->L[0] > g->L[1] ? g->L[0] : g->L[1];
  if (g->ndim == 3 && g->L[2] > Lm) Lm = g->L[2];
  const double eta = eta_ve(g);
  const double Re = g->xi * 3.0 * sqrt(10.0) * M_PI / 2.0, r = g->r_pt;
  const double Vp = g->c_cfl * dx_min(g);
  q.rho = Re * eta / (Vp * Lm);
  q.Gt = q.rho * Vp * Vp / (r + 4.0 / 3.0);
  q.Kt = r * q.Gt;
  q.beta_tau = (1.0 / (2.0 * q.Gt)) / (1.0 / (2.0 * q.Gt) + 1.0 / (2.0 * eta));
  q.beta_p = (1.0 / q.Kt) / (1.0 / q.Kt + 1.0 / (g->K * g->dt));
  q.vstep = 1.0 / q.rho;
  return q;
}

/* ------------------------------------------------------------------------ */
/* Step 4: one pseudo step of Eqs. A2ssP and A23ssP followed by the return   */
/* of Sec. 3.3.  bt = bp = 0 gives the physical (pseudo-steady) response.    */
/* ------------------------------------------------------------------------ */
static void pt_stress(or_grid *g, double bt, double bp) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  long nc = n_centres(g);
  if (!g->incompressible) {
    /* pressure, Eq. A2ssP: p = bp p_k + (1 - bp) (p_hat - K dt div v) */
    #pragma omp parallel for schedule(static)
    for (long c = 0; c < nc; ++c)
      g->pc[c] = bp * g->p_k[c] + (1.0 - bp) * (g->p[c] - g->K * g->dt * g->div[c]);
  } else if (bt != 0.0 || bp != 0.0) {
    /* pressure, Eq. A2ssP2 with pseudo step 1: p = p_k - K~ div v */
    const double Kt = pt_params(g).Kt;
    #pragma omp parallel for schedule(static)
    for (long c = 0; c < nc; ++c) g->pc[c] = g->p_k[c] - Kt * g->div[c];
  } else {
    /* the physical response: the pressure is no function of v here, it
     * keeps its old value */
    memcpy(g->pc, g->p, sizeof(double) * nc);
  }
  /* relaxed trial deviator, Eq. A23ssP: T = bt tau_k + (1 - bt) tau_tr */
  #pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c)
    for (int d = 0; d < g->ndim; ++d) g->Tn[d][c] = bt * g->tn_k[d][c] + (1.0 - bt) * g->trn[d][c];
  for (int s = 0; s < n_shear_comp(g); ++s) {
    long ns = n_shear(g, s);
    #pragma omp parallel for schedule(static)
    for (long e = 0; e < ns; ++e) g->Ts[s][e] = bt * g->ts_k[s][e] + (1.0 - bt) * g->trs[s][e];
  }
  /* Drucker-Prager return at centres (Eqs. A61, A611, A6121lambda) */
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
    long c = CI(i, j, k);
    double Txy = 0.25 * (g->Ts[0][XYI(i, j, k)] + g->Ts[0][XYI(i + 1, j, k)] +
                         g->Ts[0][XYI(i, j + 1, k)] + g->Ts[0][XYI(i + 1, j + 1, k)]);
    double J2 = Txy * Txy;
    for (int d = 0; d < g->ndim; ++d) J2 += 0.5 * g->Tn[d][c] * g->Tn[d][c];
    if (g->ndim == 3) {
      double Txz = 0.25 * (g->Ts[1][XZI(i, j, k)] + g->Ts[1][XZI(i + 1, j, k)] +
                           g->Ts[1][XZI(i, j, k + 1)] + g->Ts[1][XZI(i + 1, j, k + 1)]);
      double Tyz = 0.25 * (g->Ts[2][YZI(i, j, k)] + g->Ts[2][YZI(i, j + 1, k)] +
                           g->Ts[2][YZI(i, j, k + 1)] + g->Ts[2][YZI(i, j + 1, k + 1)]);
      J2 += Txz * Txz + Tyz * Tyz;
    }
    double sj = sqrt(J2);
    double Y = g->A * g->pc[c] + g->B * g->coh[c];
    if (Y < 0.0) Y = 0.0;
    if (!g->frozen) g->s[c] = sj > Y ? Y / sj : 1.0;
    for (int d = 0; d < g->ndim; ++d) g->sn[d][c] = g->s[c] * g->Tn[d][c];
  }
  /* vertices / edges: arithmetic mean of the adjacent centre scales */
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k) for (int j = 0; j <= ny; ++j) for (int i = 0; i <= nx; ++i) {
    long e = XYI(i, j, k);
    if (i == 0 || i == nx || j == 0 || j == ny) { g->ss[0][e] = 0.0; continue; }
    double sb = 0.25 * (g->s[CI(i - 1, j - 1, k)] + g->s[CI(i, j - 1, k)] + g->s[CI(i - 1, j, k)] + g->s[CI(i, j, k)]);
    g->ss[0][e] = sb * g->Ts[0][e];
  }
  if (g->ndim == 2) return;
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k <= nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i <= nx; ++i) {
    long e = XZI(i, j, k);
    if (i == 0 || i == nx || k == 0 || k == nz) { g->ss[1][e] = 0.0; continue; }
    double sb = 0.25 * (g->s[CI(i - 1, j, k - 1)] + g->s[CI(i, j, k - 1)] + g->s[CI(i - 1, j, k)] + g->s[CI(i, j, k)]);
    g->ss[1][e] = sb * g->Ts[1][e];
  }
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k <= nz; ++k) for (int j = 0; j <= ny; ++j) for (int i = 0; i < nx; ++i) {
    long e = YZI(i, j, k);
    if (j == 0 || j == ny || k == 0 || k == nz) { g->ss[2][e] = 0.0; continue; }
    double sb = 0.25 * (g->s[CI(i, j - 1, k - 1)] + g->s[CI(i, j, k - 1)] + g->s[CI(i, j - 1, k)] + g->s[CI(i, j, k)]);
    g->ss[2][e] = sb * g->Ts[2][e];
  }
}

/* ------------------------------------------------------------------------ */
/* Step 5: momentum residual at interior faces (Eq. A22S + body force)       */
/* ------------------------------------------------------------------------ */
static void residual(or_grid *g) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  const double dx = g->dx, dy = g->dy, dz = g->dz;
  double *sxy = g->ss[0], *sxz = g->ss[1], *syz = g->ss[2];
  const int d3 = g->ndim == 3;
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i <= nx; ++i) {
    long fi = FXI(i, j, k);
    if (i == 0 || i == nx) { g->R[0][fi] = 0.0; continue; }
    double r = ((g->sn[0][CI(i, j, k)] - g->pc[CI(i, j, k)]) - (g->sn[0][CI(i - 1, j, k)] - g->pc[CI(i - 1, j, k)])) / dx +
               (sxy[XYI(i, j + 1, k)] - sxy[XYI(i, j, k)]) / dy;
    if (d3) r += (sxz[XZI(i, j, k + 1)] - sxz[XZI(i, j, k)]) / dz;
    g->R[0][fi] = r + g->f[0][fi];
  }
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k) for (int j = 0; j <= ny; ++j) for (int i = 0; i < nx; ++i) {
    long fi = FYI(i, j, k);
    if (j == 0 || j == ny) { g->R[1][fi] = 0.0; continue; }
    double r = ((g->sn[1][CI(i, j, k)] - g->pc[CI(i, j, k)]) - (g->sn[1][CI(i, j - 1, k)] - g->pc[CI(i, j - 1, k)])) / dy +
               (sxy[XYI(i + 1, j, k)] - sxy[XYI(i, j, k)]) / dx;
    if (d3) r += (syz[YZI(i, j, k + 1)] - syz[YZI(i, j, k)]) / dz;
    g->R[1][fi] = r + g->f[1][fi];
  }
  if (!d3) return;
  #pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k <= nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
    long fi = FZI(i, j, k);
    if (k == 0 || k == nz) { g->R[2][fi] = 0.0; continue; }
    g->R[2][fi] = ((g->sn[2][CI(i, j, k)] - g->pc[CI(i, j, k)]) - (g->sn[2][CI(i, j, k - 1)] - g->pc[CI(i, j, k - 1)])) / dz +
                  (sxz[XZI(i + 1, j, k)] - sxz[XZI(i, j, k)]) / dx +
                  (syz[YZI(i, j + 1, k)] - syz[YZI(i, j, k)]) / dy + g->f[2][fi];
  }
}

/* full evaluation at velocity vv with relaxation weights (bt, bp) */
static void evaluate(or_grid *g, double *const vv[3], double bt, double bp) {
  strain_rates(g, vv);
  if (g->ndim == 2) rotated_history_2d(g); else rotated_history_3d(g);
  trial(g);
  pt_stress(g, bt, bp);
  residual(g);
  g->evaluated = 1;
}

/* copy the freshly evaluated stresses into the pseudo-time state */
static void accept_stress(or_grid *g) {
  long nc = n_centres(g);
  memcpy(g->p_k, g->pc, sizeof(double) * nc);
  for (int d = 0; d < g->ndim; ++d) memcpy(g->tn_k[d], g->sn[d], sizeof(double) * nc);
  for (int s = 0; s < n_shear_comp(g); ++s) memcpy(g->ts_k[s], g->ss[s], sizeof(double) * n_shear(g, s));
}

/* ------------------------------------------------------------------------ */
/* Advection of the old stress: the v_k d sigma_ij / dx_k part of the        */
/* Jaumann rate (Eq. j1).  The paper gives no discretisation; this reading:  */
/* once per increment, before its iteration, every history component f      */
/* (tau_hat at centres and at vertices/edges, p_hat at centres) becomes      */
/*     f - dt * sum_e v_e(x_f) * D_e f                                        */
/* with the previous increment's converged velocity v.  D_e is the upwind    */
/* one-sided difference: (f[q] - f[q-1]) / h_e where v_e > 0, (f[q+1] -      */
/* f[q]) / h_e where v_e < 0, and 0 where that neighbour lies outside the    */
/* field (an inflow wall: zero gradient).  v_e(x_f) is the arithmetic mean   */
/* of the nearest values of face component e: one value in each dimension   */
/* where the field point and face e are staggered alike, the two neighbours */
/* in each dimension where they are not.  Wall vertices/edges keep their    */
/* zero shear stress (free slip).                                            */
/* ------------------------------------------------------------------------ */

/* staggering of a field point per dimension: 1 = on cell faces/vertices,
 * 0 = at cell centres.  loc: -1 centres, c >= 0 shear component c. */
static void stagger_of(const or_grid *g, int loc, int st[3]) {
  st[0] = st[1] = st[2] = 0;
  if (loc < 0) return;
  if (g->ndim == 2) { st[0] = st[1] = 1; return; }
  st[0] = loc != 2; st[1] = loc != 1; st[2] = loc != 0;
}

/* velocity component e at point (i, j, k) of staggering st */
static double velocity_at(const or_grid *g, int e, const int st[3], int i, int j, int k) {
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int d = 0; d < g->ndim; ++d) {
    const int face_st = d == e;          /* face e sits on the grid lines of dimension e only */
    if (face_st == st[d]) continue;
    if (st[d]) { lo[d] = -1; hi[d] = 0; }  /* a grid line between cells q-1 and q */
    else { lo[d] = 0; hi[d] = 1; }         /* a centre between grid lines q and q+1 */
  }
  int ex, ey, ez; face_dims(g, e, &ex, &ey, &ez);
  double sum = 0.0;
  int cnt = 0;
  for (int c = lo[2]; c <= hi[2]; ++c)
    for (int b = lo[1]; b <= hi[1]; ++b)
      for (int a = lo[0]; a <= hi[0]; ++a) {
        sum += g->v[e][((long)(k + c) * ey + (j + b)) * ex + (i + a)];
        ++cnt;
      }
  return sum / cnt;
}

/* one field of extent (ex, ey, ez) and staggering st: out = advected f */
static void advect_field(const or_grid *g, const double *f, double *out, int ex, int ey, int ez,
                         const int st[3], double dt) {
  const double h[3] = {g->dx, g->dy, g->dz};
  const int ext[3] = {ex, ey, ez}, n[3] = {g->nx, g->ny, g->nz};
  for (int k = 0; k < ez; ++k) for (int j = 0; j < ey; ++j) for (int i = 0; i < ex; ++i) {
    const long id = ((long)k * ey + j) * ex + i;
    const int q[3] = {i, j, k};
    int wall = 0;
    for (int d = 0; d < g->ndim; ++d) if (st[d] && (q[d] == 0 || q[d] == n[d])) wall = 1;
    if (wall) { out[id] = f[id]; continue; }
    double adv = 0.0;
    for (int e = 0; e < g->ndim; ++e) {
      const double ve = velocity_at(g, e, st, i, j, k);
      const long step = e == 0 ? 1 : e == 1 ? ex : (long)ex * ey;
      double D = 0.0;
      if (ve > 0.0 && q[e] - 1 >= 0) D = (f[id] - f[id - step]) / h[e];
      else if (ve < 0.0 && q[e] + 1 < ext[e]) D = (f[id + step] - f[id]) / h[e];
      adv += ve * D;
    }
    out[id] = f[id] - dt * adv;
  }
}

/* advect tau_hat and p_hat over dt with the velocity held in g->v */
static int advect_history(or_grid *g, double dt) {
  int st[3];
  const long nc = n_centres(g);
  long nmax = nc;
  for (int c = 0; c < n_shear_comp(g); ++c) if (n_shear(g, c) > nmax) nmax = n_shear(g, c);
  double *tmp = zalloc(nmax);
  if (!tmp) return OR_ERR_OOM;
  stagger_of(g, -1, st);
  for (int d = 0; d <= g->ndim; ++d) {      /* normal components, then the pressure */
    double *f = d < g->ndim ? g->tn[d] : g->p;
    advect_field(g, f, tmp, g->nx, g->ny, g->nz, st, dt);
    memcpy(f, tmp, sizeof(double) * nc);
  }
  for (int c = 0; c < n_shear_comp(g); ++c) {
    int ex, ey, ez; shear_dims(g, c, &ex, &ey, &ez);
    stagger_of(g, c, st);
    advect_field(g, g->ts[c], tmp, ex, ey, ez, st, dt);
    memcpy(g->ts[c], tmp, sizeof(double) * n_shear(g, c));
  }
  free(tmp);
  return OR_OK;
}

/* Incompressible variant (Sec. 3.2, Eq. A2ssP2): the pressure equation
 * (1/K~) dp/dt~ = -div v replaces Eq. A2ssP; K is not used.  The pressure is
 * pseudo-time state that starts at p_hat (no function of v gives it), and
 * its stopping measure is 2 eta_ve <|div v|> / max|sigma|: the volumetric
 * rate error in the stress units of the deviatoric response. */
int or_set_incompressible(or_grid *g, int on) {
  g->incompressible = on != 0;
  return OR_OK;
}

/* Per-cell shear modulus (one positive value per centre, copied; NULL
 * returns to the uniform G of or_set_material).  eta_ve and the weight of
 * the rotated old stress then vary point by point (vertices/edges: mean of
 * the adjacent centres); the pseudo-transient parameters use the largest G,
 * which changes the iteration count but not the fixed point. */
int or_set_shear_modulus(or_grid *g, const double *Gc) {
  if (!Gc) { free(g->Gc); g->Gc = NULL; return OR_OK; }
  const long nc = n_centres(g);
  double mx = 0.0;
  for (long c = 0; c < nc; ++c) {
    if (!(Gc[c] > 0.0) || isinf(Gc[c])) return OR_ERR_ARG;
    if (Gc[c] > mx) mx = Gc[c];
  }
  if (!g->Gc) g->Gc = zalloc(nc);
  if (!g->Gc) return OR_ERR_OOM;
  memcpy(g->Gc, Gc, sizeof(double) * nc);
  g->Gref = mx;
  return OR_OK;
}

/* Switch the per-increment advection of the old stress on or off. */
int or_set_advection(or_grid *g, int on) {
  g->advect = on != 0;
  return OR_OK;
}

/* Advect the history now over dt with the velocity field g->v (the step
 * or_apply_increment takes when advection is on). */
int or_advect(or_grid *g, double dt) {
  if (!(dt >= 0.0)) return OR_ERR_ARG;
  return advect_history(g, dt);
}

/* Start of an increment (A0): the walls get the velocities of the pure-shear
 * (or any diagonal) background gradient, v_d = rate[d] * x_d (Eqs. A7-A9M);
 * the interior starts from the last converged field, or from the background
 * field on the first increment.  f (nullable) is the body force at the faces,
 * one array per component, concatenated x, y[, z].  The pseudo-time stress
 * state starts at the physical response to the start velocity. */
int or_apply_increment(or_grid *g, const double *rate, double dt, const double *f) {
  if (!g->have_material || !(dt > 0.0)) return OR_ERR_ARG;
  for (int d = 0; d < 3; ++d) g->rate[d] = d < g->ndim ? rate[d] : 0.0;
  g->dt = dt;
  if (g->advect && g->commits > g->adv_done) {   /* once per committed increment */
    int r = advect_history(g, dt);
    if (r != OR_OK) return r;
    g->adv_done = g->commits;
  }
  long off = 0;
  for (int d = 0; d < g->ndim; ++d) {
    long nf = n_face(g, d);
    if (f) memcpy(g->f[d], f + off, sizeof(double) * nf); else memset(g->f[d], 0, sizeof(double) * nf);
    off += nf;
    int ex, ey, ez; face_dims(g, d, &ex, &ey, &ez);
    for (int k = 0; k < ez; ++k) for (int j = 0; j < ey; ++j) for (int i = 0; i < ex; ++i) {
      long id = ((long)k * ey + j) * ex + i;
      int c = d == 0 ? i : d == 1 ? j : k;
      double vb = g->rate[d] * (-0.5 * g->L[d] + c * spacing(g, d));
      if (is_boundary_face(g, d, i, j, k) || !g->started) g->v0[d][id] = vb;
      else g->v0[d][id] = g->v[d][id];
    }
  }
  g->started = 1;
  g->in_increment = 1;
  g->evaluated = 0;
  return OR_OK;
}

/* Replace the interior start velocity (e.g. a predicted start); walls keep
 * the prescribed values. */
int or_set_start(or_grid *g, const double *v) {
  if (!g->in_increment) return OR_ERR_STATE;
  long off = 0;
  for (int d = 0; d < g->ndim; ++d) {
    int ex, ey, ez; face_dims(g, d, &ex, &ey, &ez);
    for (int k = 0; k < ez; ++k) for (int j = 0; j < ey; ++j) for (int i = 0; i < ex; ++i) {
      long id = ((long)k * ey + j) * ex + i;
      if (!is_boundary_face(g, d, i, j, k)) g->v0[d][id] = v[off + id];
    }
    off += n_face(g, d);
  }
  return OR_OK;
}

/* L-infinity norms (Eq. Convergence1) of the last evaluation: max|R|,
 * max|sigma|, and the largest change of the deviator and of the pressure
 * since the previous check (the stress state saved then).  When `refresh`
 * is set the saved state becomes the new one. */
static void norms(or_grid *g, double *max_r, double *max_sig, double *d_tau, double *d_p, int refresh) {
  double mr = 0.0, ms = 0.0, dtau = 0.0, dp = 0.0;
  int nan_seen = 0;
  for (int d = 0; d < g->ndim; ++d) {
    long nf = n_face(g, d);
    for (long i = 0; i < nf; ++i) {
      double a = fabs(g->R[d][i]);
      if (a != a) nan_seen = 1; else if (a > mr) mr = a;
    }
  }
  long nc = n_centres(g);
  for (long c = 0; c < nc; ++c) {
    for (int d = 0; d < g->ndim; ++d) {
      double a = fabs(g->sn[d][c] - g->pc[c]); if (a > ms) ms = a;
      double b = fabs(g->sn[d][c] - g->tn_c[d][c]); if (b > dtau) dtau = b;
      if (refresh) g->tn_c[d][c] = g->sn[d][c];
    }
    double b = fabs(g->pc[c] - g->p_c[c]); if (b > dp) dp = b;
    if (refresh) g->p_c[c] = g->pc[c];
  }
  for (int s = 0; s < n_shear_comp(g); ++s) {
    long ns = n_shear(g, s);
    for (long e = 0; e < ns; ++e) {
      double a = fabs(g->ss[s][e]); if (a > ms) ms = a;
      double b = fabs(g->ss[s][e] - g->ts_c[s][e]); if (b > dtau) dtau = b;
      if (refresh) g->ts_c[s][e] = g->ss[s][e];
    }
  }
  if (nan_seen) mr = NAN;
  *max_r = mr; *max_sig = ms; *d_tau = dtau; *d_p = dp;
}

/* copy the pseudo-time stress state into the check snapshot */
static void snapshot_state(or_grid *g) {
  long nc = n_centres(g);
  memcpy(g->p_c, g->p_k, sizeof(double) * nc);
  for (int d = 0; d < g->ndim; ++d) memcpy(g->tn_c[d], g->tn_k[d], sizeof(double) * nc);
  for (int s = 0; s < n_shear_comp(g); ++s) memcpy(g->ts_c[s], g->ts_k[s], sizeof(double) * n_shear(g, s));
}

static void diagnostics(or_grid *g, or_info *info) {
  long np = 0;
  for (long c = 0; c < n_centres(g); ++c) np += g->s[c] < 1.0;
  info->n_plastic = np;
  /* integrated sigma_xx along the vertical centre line and the rightmost
   * column (2D: sum over j of sigma_xx dy; 3D: sum over k dz at j = ny/2) */
  double a = 0.0, b = 0.0;
  int ic = g->nx / 2, ir = g->nx - 1;
  if (g->ndim == 2) {
    for (int j = 0; j < g->ny; ++j) {
      a += (g->sn[0][CI(ic, j, 0)] - g->pc[CI(ic, j, 0)]) * g->dy;
      b += (g->sn[0][CI(ir, j, 0)] - g->pc[CI(ir, j, 0)]) * g->dy;
    }
  } else {
    int jc = g->ny / 2;
    for (int k = 0; k < g->nz; ++k) {
      a += (g->sn[0][CI(ic, jc, k)] - g->pc[CI(ic, jc, k)]) * g->dz;
      b += (g->sn[0][CI(ir, jc, k)] - g->pc[CI(ir, jc, k)]) * g->dz;
    }
  }
  info->sxx_int_centre = a; info->sxx_int_right = b;
}

/* The pseudo-transient iteration for one increment.  State (v_k, tau_k, p_k)
 * starts at (v0, physical response to v0).  Iteration k:
 *   1. p_{k+1}, tau_{k+1} from one pseudo step of Eqs. A2ssP/A23ssP and the
 *      return, using v_k;
 *   2. R_k = div(tau_{k+1} - p_{k+1} I) + f (Eq. A22S);
 *   3. at k = 0 and every n_chk-th k, with m the iterations since the previous
 *      check (m = 1 at k = 0, whose reference state is the start state):
 *      eps_mom = dx_min max|v_{k+1} - v_chk| rho~ / m / max|sigma| (the
 *      momentum residual averaged over the interval; v_{k+1} = v_k + R_k/rho~),
 *      eps_tau = max|tau_{k+1} - tau_chk| / (m (1 - beta_tau)) / max|sigma|,
 *      eps_p = max|p_{k+1} - p_chk| / (m (1 - beta_p)) / max|sigma|
 *      (each equation's residual in stress units, the pseudo-time rates taken
 *      over the check interval as eps_rel takes V - V^it, Eq. Convergence2),
 *      eps_res = the largest; stop when eps_res <= tol, keeping
 *      (v_k, tau_{k+1}, p_{k+1});
 *   4. v_{k+1} = v_k + R_k / rho~ at interior faces (Eq. A22P).
 * With frozen plasticity enabled, a check that does not stop and has
 * k >= freeze_iter and eps_rel > freeze_eps freezes the centre scales s of
 * iteration k for all later iterations of the increment. */
int or_solve_increment(or_grid *g, or_info *info) {
  if (!g->in_increment) return OR_ERR_STATE;
  memset(info, 0, sizeof(*info));
  const pt_t q = pt_params(g);
  for (int d = 0; d < g->ndim; ++d) {
    long nf = n_face(g, d);
    memcpy(g->vi[d], g->v0[d], sizeof(double) * nf);
    memcpy(g->vchk[d], g->v0[d], sizeof(double) * nf);
  }
  /* start stress: physical response to v0 */
  evaluate(g, g->vi, 0.0, 0.0);
  accept_stress(g);
  snapshot_state(g);
  const double dxm = dx_min(g);
  int status = OR_ERR_NOT_CONVERGED;
  long k_prev = -1;
  g->frozen = 0;
  info->frozen_at = -1;
  for (long k = 0;; ++k) {
    evaluate(g, g->vi, q.beta_tau, q.beta_p);
    if (k % g->n_chk == 0 || k == g->max_iter) {
      double mr, ms, dtau, dp;
      norms(g, &mr, &ms, &dtau, &dp, 1);
      const double m = (double)(k - k_prev);
      k_prev = k;
      /* velocity after this iteration's update, compared with the one after
       * the previous check's update: the momentum residual averaged over the
       * check interval is rho~ (v_{k+1} - v_chk) / m (Eq. A22P) */
      double dvm = 0.0, vm = 0.0;
      for (int d = 0; d < g->ndim; ++d) {
        int ex, ey, ez; face_dims(g, d, &ex, &ey, &ez);
        for (int kk = 0; kk < ez; ++kk) for (int j = 0; j < ey; ++j) for (int i = 0; i < ex; ++i) {
          long id = ((long)kk * ey + j) * ex + i;
          double vn = g->vi[d][id];
          if (!is_boundary_face(g, d, i, j, kk)) vn = g->vi[d][id] + q.vstep * g->R[d][id];
          double a = fabs(vn - g->vchk[d][id]); if (a > dvm || a != a) dvm = a;
          double b = fabs(g->vi[d][id]); if (b > vm) vm = b;
          g->vchk[d][id] = vn;
        }
      }
      double em = (dvm == 0.0) ? 0.0 : (ms > 0.0 ? dxm * dvm / (m * q.vstep) / ms : INFINITY);
      double et = (dtau == 0.0) ? 0.0 : (ms > 0.0 ? dtau / (m * (1.0 - q.beta_tau)) / ms : INFINITY);
      /* pressure measure: the distance of p from its target (compressible);
       * incompressible, 2 eta_ve times the interval-averaged divergence
       * (p_{k+1} - p_chk = -K~ m <div v>) */
      double ep = (dp == 0.0) ? 0.0
                  : !(ms > 0.0) ? INFINITY
                  : g->incompressible ? 2.0 * eta_ve(g) * dp / (m * q.Kt) / ms
                                      : dp / (m * (1.0 - q.beta_p)) / ms;
      double er = em > et ? em : et;
      if (ep > er) er = ep;
      info->iters = k; info->eps_res = er; info->eps_mom = em; info->eps_tau = et; info->eps_p = ep;
      info->max_r = mr; info->max_sigma = ms;
      info->eps_rel = vm > 0.0 ? dvm / vm : 0.0;
      if (mr != mr || er != er) { status = OR_ERR_DIVERGED; break; }
      if (er <= g->tol) { status = OR_OK; break; }
      if (k >= g->max_iter) break;
      if (!g->frozen && g->freeze_iter > 0 && k >= g->freeze_iter && info->eps_rel > g->freeze_eps) {
        g->frozen = 1;
        info->frozen_at = k;
      }
    }
    /* accept the new stress state and update interior velocities (A22P) */
    accept_stress(g);
    for (int d = 0; d < g->ndim; ++d) {
      int ex, ey, ez; face_dims(g, d, &ex, &ey, &ez);
#pragma omp parallel for collapse(2) schedule(static)
      for (int kk = 0; kk < ez; ++kk) for (int j = 0; j < ey; ++j) for (int i = 0; i < ex; ++i) {
        if (is_boundary_face(g, d, i, j, kk)) continue;
        long id = ((long)kk * ey + j) * ex + i;
        g->vi[d][id] += q.vstep * g->R[d][id];
      }
    }
  }
  g->frozen = 0;   /* the scales of this solve stay in g->s for the commit */
  info->status = status;
  diagnostics(g, info);
  return status;
}

/* Evaluate at a caller-given face velocity (concatenated x, y[, z], walls
 * included) with the physical response (no pseudo-time memory): the stress
 * and residual of the fixed point at v.  Returns max|R| and max|sigma|. */
/* Threads of the per-iteration loops: n > 0 sets their number; returns the
 * number in use (1 in a build without OpenMP). */
int or_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int or_eval(or_grid *g, const double *v, double *max_r, double *max_sig) {
  if (!g->in_increment) return OR_ERR_STATE;
  long off = 0;
  for (int d = 0; d < g->ndim; ++d) { long nf = n_face(g, d); memcpy(g->vi[d], v + off, sizeof(double) * nf); off += nf; }
  evaluate(g, g->vi, 0.0, 0.0);
  accept_stress(g);
  double dtau, dp;
  norms(g, max_r, max_sig, &dtau, &dp, 0);
  return OR_OK;
}

/* The stress of the last evaluation (or_eval gives the physical response of
 * a velocity): comp 0..2 the centre deviator components, 3..5 the shear
 * components (vertices/edges), 6 the pressure. */
int or_get_eval(or_grid *g, int comp, double *out, long count) {
  if (!g->evaluated || comp < 0 || comp > 6) return OR_ERR_STATE;
  const double *src;
  long n;
  if (comp < 3) {
    if (comp >= g->ndim) return OR_ERR_ARG;
    src = g->sn[comp]; n = n_centres(g);
  } else if (comp < 6) {
    if (comp - 3 >= n_shear_comp(g)) return OR_ERR_ARG;
    src = g->ss[comp - 3]; n = n_shear(g, comp - 3);
  } else {
    src = g->pc; n = n_centres(g);
  }
  if (count != n) return OR_ERR_ARG;
  memcpy(out, src, sizeof(double) * n);
  return OR_OK;
}

/* A9 history commit from the last evaluation at the converged iterate:
 * tau_hat <- tau, p_hat <- p; at centres where the return acted (s < 1) the
 * plastic strain grows by dt times the magnitude sqrt(J2) of the plastic
 * strain rate (tau_tr - tau) / (2 eta_ve) (Eq. A23ssP at pseudo-steady state;
 * shear parts averaged to the centre);
 * displacement and accumulated strain grow by dt times the rates; the
 * converged velocity becomes the iterate. */
int or_commit(or_grid *g) {
  if (!g->in_increment || !g->evaluated) return OR_ERR_STATE;
  const double dt = g->dt;
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  for (int k = 0; k < nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
    long c = CI(i, j, k);
    double J2 = 0.0;
    for (int d = 0; d < g->ndim; ++d) { double a = g->trn[d][c] - g->sn[d][c]; J2 += 0.5 * a * a; }
    double a = 0.25 * ((g->trs[0][XYI(i, j, k)] - g->ss[0][XYI(i, j, k)]) + (g->trs[0][XYI(i + 1, j, k)] - g->ss[0][XYI(i + 1, j, k)]) +
                       (g->trs[0][XYI(i, j + 1, k)] - g->ss[0][XYI(i, j + 1, k)]) + (g->trs[0][XYI(i + 1, j + 1, k)] - g->ss[0][XYI(i + 1, j + 1, k)]));
    J2 += a * a;
    if (g->ndim == 3) {
      double b = 0.25 * ((g->trs[1][XZI(i, j, k)] - g->ss[1][XZI(i, j, k)]) + (g->trs[1][XZI(i + 1, j, k)] - g->ss[1][XZI(i + 1, j, k)]) +
                         (g->trs[1][XZI(i, j, k + 1)] - g->ss[1][XZI(i, j, k + 1)]) + (g->trs[1][XZI(i + 1, j, k + 1)] - g->ss[1][XZI(i + 1, j, k + 1)]));
      double cc = 0.25 * ((g->trs[2][YZI(i, j, k)] - g->ss[2][YZI(i, j, k)]) + (g->trs[2][YZI(i, j + 1, k)] - g->ss[2][YZI(i, j + 1, k)]) +
                          (g->trs[2][YZI(i, j, k + 1)] - g->ss[2][YZI(i, j, k + 1)]) + (g->trs[2][YZI(i, j + 1, k + 1)] - g->ss[2][YZI(i, j + 1, k + 1)]));
      J2 += b * b + cc * cc;
    }
    if (g->s[c] < 1.0) g->epl[c] += dt * sqrt(J2) / (2.0 * eta_for(g, G_centre(g, c)));   /* only where the return acted */
  }
  long nc = n_centres(g);
  for (long c = 0; c < nc; ++c) {
    for (int d = 0; d < g->ndim; ++d) {
      g->tn[d][c] = g->sn[d][c];
      g->an[d][c] += dt * g->en[d][c];
    }
    g->p[c] = g->pc[c];
  }
  for (int s = 0; s < n_shear_comp(g); ++s) {
    long ns = n_shear(g, s);
    for (long e = 0; e < ns; ++e) { g->ts[s][e] = g->ss[s][e]; g->as[s][e] += dt * g->es[s][e]; }
  }
  for (int d = 0; d < g->ndim; ++d) {
    long nf = n_face(g, d);
    for (long i = 0; i < nf; ++i) { g->v[d][i] = g->vi[d][i]; g->u[d][i] += dt * g->vi[d][i]; }
  }
  g->in_increment = 0;
  g->commits += 1;
  return OR_OK;
}

/* ---------------- field access (compact FP64 arrays, x fastest) ---------- */
static long field_count(const or_grid *g, int f) {
  switch (f) {
    case OF_VX: case OF_UX: case OF_V0X: case OF_RX: return n_face(g, 0);
    case OF_VY: case OF_UY: case OF_V0Y: case OF_RY: return n_face(g, 1);
    case OF_VZ: case OF_UZ: case OF_V0Z: case OF_RZ: return g->ndim == 3 ? n_face(g, 2) : 0;
    case OF_TXX: case OF_TYY: case OF_P: case OF_EPL: case OF_EXX: case OF_EYY:
    case OF_COH: case OF_EII: case OF_SCALE: return n_centres(g);
    case OF_TZZ: case OF_EZZ: return g->ndim == 3 ? n_centres(g) : 0;
    case OF_TXY: case OF_EXY: return n_shear(g, 0);
    case OF_TXZ: case OF_EXZ: return g->ndim == 3 ? n_shear(g, 1) : 0;
    case OF_TYZ: case OF_EYZ: return g->ndim == 3 ? n_shear(g, 2) : 0;
    default: return -1;
  }
}

static double *field_ptr(or_grid *g, int f) {
  switch (f) {
    case OF_VX: return g->v[0]; case OF_VY: return g->v[1]; case OF_VZ: return g->v[2];
    case OF_TXX: return g->tn[0]; case OF_TYY: return g->tn[1]; case OF_TZZ: return g->tn[2];
    case OF_TXY: return g->ts[0]; case OF_TXZ: return g->ts[1]; case OF_TYZ: return g->ts[2];
    case OF_P: return g->p; case OF_EPL: return g->epl;
    case OF_UX: return g->u[0]; case OF_UY: return g->u[1]; case OF_UZ: return g->u[2];
    case OF_EXX: return g->an[0]; case OF_EYY: return g->an[1]; case OF_EZZ: return g->an[2];
    case OF_EXY: return g->as[0]; case OF_EXZ: return g->as[1]; case OF_EYZ: return g->as[2];
    case OF_COH: return g->coh; case OF_SCALE: return g->s;
    case OF_V0X: return g->v0[0]; case OF_V0Y: return g->v0[1]; case OF_V0Z: return g->v0[2];
    case OF_RX: return g->R[0]; case OF_RY: return g->R[1]; case OF_RZ: return g->R[2];
    default: return NULL;
  }
}

long or_field_count(or_grid *g, int f) { return field_count(g, f); }

int or_get_field(or_grid *g, int f, double *out, long count) {
  long n = field_count(g, f);
  if (n < 0 || count != n) return OR_ERR_ARG;
  if (f == OF_EII) {
    /* eps_II = sqrt(eps:eps / 2) of the accumulated total strain, shear
     * components averaged from the 4 surrounding vertices/edges */
    for (int k = 0; k < g->nz; ++k) for (int j = 0; j < g->ny; ++j) for (int i = 0; i < g->nx; ++i) {
      long c = CI(i, j, k);
      double sq = 0.0;
      for (int d = 0; d < g->ndim; ++d) sq += 0.5 * g->an[d][c] * g->an[d][c];
      double exy = 0.25 * (g->as[0][XYI(i, j, k)] + g->as[0][XYI(i + 1, j, k)] + g->as[0][XYI(i, j + 1, k)] + g->as[0][XYI(i + 1, j + 1, k)]);
      sq += exy * exy;
      if (g->ndim == 3) {
        double exz = 0.25 * (g->as[1][XZI(i, j, k)] + g->as[1][XZI(i + 1, j, k)] + g->as[1][XZI(i, j, k + 1)] + g->as[1][XZI(i + 1, j, k + 1)]);
        double eyz = 0.25 * (g->as[2][YZI(i, j, k)] + g->as[2][YZI(i, j + 1, k)] + g->as[2][YZI(i, j, k + 1)] + g->as[2][YZI(i, j + 1, k + 1)]);
        sq += exz * exz + eyz * eyz;
      }
      out[c] = sqrt(sq);
    }
    return OR_OK;
  }
  double *p = field_ptr(g, f);
  if (!p) return OR_ERR_ARG;
  memcpy(out, p, sizeof(double) * n);
  return OR_OK;
}

/* Set a history field (for resume tests). */
int or_set_field(or_grid *g, int f, const double *in, long count) {
  long n = field_count(g, f);
  if (n < 0 || count != n || f == OF_EII || f == OF_SCALE || f == OF_RX || f == OF_RY || f == OF_RZ ||
      f == OF_V0X || f == OF_V0Y || f == OF_V0Z) return OR_ERR_ARG;
  double *p = field_ptr(g, f);
  if (!p) return OR_ERR_ARG;
  memcpy(p, in, sizeof(double) * n);
  if (f == OF_VX || f == OF_VY || f == OF_VZ) g->started = 1;
  return OR_OK;
}

/* beta_tau, beta_p and the velocity step of the current increment */
void or_pt_params(or_grid *g, double *bt, double *bp, double *vstep) {
  pt_t q = pt_params(g);
  *bt = q.beta_tau; *bp = q.beta_p; *vstep = q.vstep;
}
