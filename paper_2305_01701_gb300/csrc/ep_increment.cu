// ep_increment.cu -- FP64 kernels run once per load increment: the start
// velocity (walls from the pure-shear gradient, Eqs. A7-A9M), the rotation
// coefficients of the old stress (Eq. j14, Appendix A), the history commit
// (the "old" fields of Fig. 1) and field packing for the host interface.
#include <math.h>

#include "ep_internal.cuh"

namespace ep {

namespace {

constexpr int kThreads = 256;

struct Pos3 {
  int i, j, k;
  long long e;
  bool in;
};

__device__ __forceinline__ Pos3 pos3(const Geo &g) {
  Pos3 p;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  p.in = t < g.box;
  p.e = t;
  p.i = (int)(t % g.px);
  long long r = t / g.px;
  p.j = (int)(r % g.py);
  p.k = (int)(r / g.py);
  return p;
}

inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// is (i,j,k) inside the extent of face component d?
__device__ __forceinline__ bool face_in(const Geo &g, int d, int i, int j, int k) {
  const int ez = g.ndim == 3 ? g.nz : 1;
  if (d == 0) return i <= g.nx && j < g.ny && k < ez;
  if (d == 1) return i < g.nx && j <= g.ny && k < ez;
  return i < g.nx && j < g.ny && k <= g.nz;
}
__device__ __forceinline__ bool face_wall(const Geo &g, int d, int i, int j, int k) {
  return d == 0 ? (i == 0 || i == g.nx) : d == 1 ? (j == 0 || j == g.ny) : (k == 0 || k == g.nz);
}

__global__ void k_start_velocity(Geo g, History H, const double *dv0, const double *dv1, const double *dv2,
                                 const Scal *sc, int started, double Lx, double Ly, double Lz) {
  const Pos3 q = pos3(g);
  if (!q.in) return;
  const double *dv[3] = {dv0, dv1, dv2};
  const double L[3] = {Lx, Ly, Lz};
  const double h[3] = {g.dx, g.dy, g.dz};
  const int c[3] = {q.i, q.j, q.k};
  for (int d = 0; d < g.ndim; ++d) {
    double v = 0.0;
    if (face_in(g, d, q.i, q.j, q.k)) {
      const double vb = sc->rate[d] * (-0.5 * L[d] + c[d] * h[d]);
      if (face_wall(g, d, q.i, q.j, q.k) || !started) v = vb;
      else v = H.v[d][q.e];
      if (dv[d] && !face_wall(g, d, q.i, q.j, q.k)) v += dv[d][q.e];
    }
    H.v0[d][q.e] = v;
  }
}

template <typename T>
__global__ void k_rotation_fields(Geo g, History H, const Scal *sc, T *rq0, T *rq1, T *rq2, T *rd0, T *rd1,
                                  T *yc) {
  const Pos3 q = pos3(g);
  if (!q.in) return;
  const int i = q.i, j = q.j, k = q.k;
  const long long e = q.e;
  const double w = sc->jaumann ? (sc->gcell ? sc->dt : sc->c2dt) : 0.0;
  const bool centre = i < g.nx && j < g.ny && (g.ndim == 2 || k < g.nz);
  if (centre) {
    rd0[e] = (T)(w * (H.tn[1][e] - H.tn[0][e]));
    if (g.ndim == 3) rd1[e] = (T)(w * (H.tn[2][e] - H.tn[0][e]));
    yc[e] = (T)(sc->B * H.coh[e]);
  } else {
    rd0[e] = (T)0;
    if (g.ndim == 3) rd1[e] = (T)0;
    yc[e] = (T)0;
  }
  rq0[e] = (T)(w * H.ts[0][e]);
  if (g.ndim == 3) {
    rq1[e] = (T)(w * H.ts[1][e]);
    rq2[e] = (T)(w * H.ts[2][e]);
  }
}

template <typename T>
__global__ void k_compose(Geo g, const double *v00, const double *v01, const double *v02, const T *u0,
                          const T *u1, const T *u2, double *o0, double *o1, double *o2) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.box) return;
  o0[t] = v00[t] + (double)u0[t];
  o1[t] = v01[t] + (double)u1[t];
  if (g.ndim == 3) o2[t] = v02[t] + (double)u2[t];
}

// History commit.  Tn64/Ts64: physical trial at the converged velocity
// H.v (already composed); es64: its shear strain rates; stn/sts/stp/s: the
// converged pseudo-time state and last return scales.
template <typename T>
__global__ void k_commit(Geo g, History H, const double *Tn0, const double *Tn1, const double *Tn2,
                         const double *Ts0, const double *Ts1, const double *Ts2, const double *es0,
                         const double *es1, const double *es2, const T *stn0, const T *stn1, const T *stn2,
                         const T *sts0, const T *sts1, const T *sts2, const T *stp, const T *s, const Scal *sc,
                         unsigned long long *n_plastic) {
  const Pos3 q = pos3(g);
  int plastic = 0;
  if (q.in) {
    const int i = q.i, j = q.j, k = q.k, nx = g.nx, ny = g.ny, nz = g.nz;
    const long long e = q.e, px = g.px, pl = g.plane;
    const double dt = sc->dt;
    const bool centre = i < nx && j < ny && (g.ndim == 2 || k < nz);
    if (centre) {
      const double Tn[3] = {Tn0[e], Tn1[e], g.ndim == 3 ? Tn2[e] : 0.0};
      const double tn[3] = {(double)stn0[e], (double)stn1[e], g.ndim == 3 ? (double)stn2[e] : 0.0};
      double J2 = 0.0;
      for (int d = 0; d < g.ndim; ++d) J2 += 0.5 * (Tn[d] - tn[d]) * (Tn[d] - tn[d]);
      double a = 0.25 * ((Ts0[e] - (double)sts0[e]) + (Ts0[e + 1] - (double)sts0[e + 1]) +
                         (Ts0[e + px] - (double)sts0[e + px]) + (Ts0[e + px + 1] - (double)sts0[e + px + 1]));
      J2 += a * a;
      if (g.ndim == 3) {
        double b = 0.25 * ((Ts1[e] - (double)sts1[e]) + (Ts1[e + 1] - (double)sts1[e + 1]) +
                           (Ts1[e + pl] - (double)sts1[e + pl]) + (Ts1[e + pl + 1] - (double)sts1[e + pl + 1]));
        double cc = 0.25 * ((Ts2[e] - (double)sts2[e]) + (Ts2[e + px] - (double)sts2[e + px]) +
                            (Ts2[e + pl] - (double)sts2[e + pl]) + (Ts2[e + pl + px] - (double)sts2[e + pl + px]));
        J2 += b * b + cc * cc;
      }
      if ((double)s[e] < 1.0) {
        H.epl[e] += dt * sqrt(J2) / (H.te_c ? H.te_c[e] : sc->two_eta);
        plastic = 1;
      }
      double ex = (H.v[0][e + 1] - H.v[0][e]) * g.rdx;
      double ey = (H.v[1][e + px] - H.v[1][e]) * g.rdy;
      H.an[0][e] += dt * ex;
      H.an[1][e] += dt * ey;
      if (g.ndim == 3) H.an[2][e] += dt * (H.v[2][e + pl] - H.v[2][e]) * g.rdz;
      for (int d = 0; d < g.ndim; ++d) H.tn[d][e] = tn[d];
      H.p[e] = (double)stp[e];
    }
    if (i <= nx && j <= ny && k <= (g.ndim == 3 ? nz : 0)) {
      H.ts[0][e] = (double)sts0[e];
      H.as[0][e] += dt * es0[e];
      if (g.ndim == 3) {
        H.ts[1][e] = (double)sts1[e];
        H.ts[2][e] = (double)sts2[e];
        H.as[1][e] += dt * es1[e];
        H.as[2][e] += dt * es2[e];
      }
    }
    for (int d = 0; d < g.ndim; ++d)
      if (face_in(g, d, i, j, k)) H.u[d][e] += dt * H.v[d][e];
  }
  // block count of plastic centres
  unsigned m = __ballot_sync(0xffffffffu, plastic);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(n_plastic, (unsigned long long)__popc(m));
}

template <typename Td, typename Ts>
__global__ void k_convert(Td *dst, const Ts *src, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = (Td)src[t];
}

// integrated sigma_xx = tau_xx - p along the centre column and the rightmost
// column (2D: sum over j of dy; 3D: sum over k of dz at j = ny/2)
__global__ void k_line_integrals(Geo g, History H, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int ic = g.nx / 2, ir = g.nx - 1, jc = g.ny / 2;
  double a = 0.0, b = 0.0;
  if (g.ndim == 2) {
    for (int j = 0; j < g.ny; ++j) {
      long long ec = g.idx(ic, j, 0), er = g.idx(ir, j, 0);
      a += (H.tn[0][ec] - H.p[ec]) * g.dy;
      b += (H.tn[0][er] - H.p[er]) * g.dy;
    }
  } else {
    for (int k = 0; k < g.nz; ++k) {
      long long ec = g.idx(ic, jc, k), er = g.idx(ir, jc, k);
      a += (H.tn[0][ec] - H.p[ec]) * g.dz;
      b += (H.tn[0][er] - H.p[er]) * g.dz;
    }
  }
  out[0] = a;
  out[1] = b;
}

__global__ void k_pack(const double *box, double *dst, int ex, int ey, int ez, int px, int py) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)ex * ey * ez;
  if (t >= n) return;
  int i = (int)(t % ex);
  long long r = t / ex;
  int j = (int)(r % ey), k = (int)(r / ey);
  dst[t] = box[((long long)k * py + j) * px + i];
}

__global__ void k_unpack(const double *src, double *box, int ex, int ey, int ez, int px, int py) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)ex * ey * ez;
  if (t >= n) return;
  int i = (int)(t % ex);
  long long r = t / ex;
  int j = (int)(r % ey), k = (int)(r / ey);
  box[((long long)k * py + j) * px + i] = src[t];
}

// Per-point Maxwell coefficients of a per-cell shear modulus G (centres):
// at centres G itself, at a vertex/edge the mean of the G of the centres
// around it (one layer along each direction in which the point sits at cell
// centres, two along the others; indices clamped at the walls); then
// 2 eta_ve = 2 / (1/(G dt) + 1/mu_s) and c2 = eta_ve / (G dt).
__global__ void k_shear_fields(Geo g, const double *Gc, double mu_s, double dt, double *ge0, double *ge1,
                               double *ge2, double *ge3, double *gc0, double *gc1, double *gc2, double *gc3) {
  const Pos3 q = pos3(g);
  if (!q.in) return;
  const int nd = g.ndim, ez = nd == 3 ? g.nz : 1;
  double *ge[4] = {ge0, ge1, ge2, ge3}, *gc[4] = {gc0, gc1, gc2, gc3};
  auto coef = [&](double G, double *a, double *b) {
    const double eta = isinf(mu_s) ? G * dt : 1.0 / (1.0 / (G * dt) + 1.0 / mu_s);
    *a = 2.0 * eta;
    *b = eta / (G * dt);
  };
  const bool centre = q.i < g.nx && q.j < g.ny && q.k < ez;
  double a = 0.0, b = 0.0;
  if (centre) coef(Gc[q.e], &a, &b);
  ge[0][q.e] = a;
  gc[0][q.e] = b;
  const int ns = nd == 3 ? 3 : 1;
  for (int c = 0; c < ns; ++c) {
    // staggering of shear component c: 1 along the directions of its faces
    const int sx = nd == 2 ? 1 : c != 2, sy = nd == 2 ? 1 : c != 1, sz = nd == 2 ? 0 : c != 0;
    double sum = 0.0;
    int cnt = 0;
    for (int dz = -sz; dz <= 0; ++dz)
      for (int dy = -sy; dy <= 0; ++dy)
        for (int dx = -sx; dx <= 0; ++dx) {
          const int i = min(max(q.i + dx, 0), g.nx - 1), j = min(max(q.j + dy, 0), g.ny - 1);
          const int k = min(max(q.k + dz, 0), ez - 1);
          sum += Gc[g.idx(i, j, k)];
          ++cnt;
        }
    a = 0.0; b = 0.0;
    const bool in = q.i <= g.nx && q.j <= g.ny && q.k <= (nd == 3 ? g.nz : 0);
    if (in) coef(sum / cnt, &a, &b);
    ge[1 + c][q.e] = a;
    gc[1 + c][q.e] = b;
  }
}

// out = scale * div(v) at centres, 0 elsewhere (the incompressible sweep's
// base pressure step -K~ div v0, Eq. A2ssP2)
__global__ void k_scaled_div(Geo g, const double *v0, const double *v1, const double *v2, double scale, double *out) {
  const Pos3 q = pos3(g);
  if (!q.in) return;
  const bool centre = q.i < g.nx && q.j < g.ny && (g.ndim == 2 || q.k < g.nz);
  double d = 0.0;
  if (centre) {
    d = (v0[q.e + 1] - v0[q.e]) * g.rdx + (v1[q.e + g.px] - v1[q.e]) * g.rdy;
    if (g.ndim == 3) d += (v2[q.e + g.plane] - v2[q.e]) * g.rdz;
  }
  out[q.e] = centre ? scale * d : 0.0;
}

// ---- advection of the old stress (the v_k d sigma_ij / dx_k term, Eq. j1) ----
// Once per increment: f <- f - dt * sum_e v_e D_e f for every history
// component, with H.v the last converged velocity.  D_e is the first-order
// upwind difference (the neighbour on the side the flow comes from; zero
// where that neighbour is outside the field).  v_e at a field point is the
// mean of the nearest face values of component e: in each dimension where
// the point and face e are staggered alike one value, otherwise the two
// neighbours.  st[d] = 1 marks a point on grid lines of dimension d.

__device__ __forceinline__ double face_mean(const Geo &g, const double *v, int e, const int st[3], int i, int j,
                                            int k) {
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int d = 0; d < g.ndim; ++d) {
    const int fs = d == e;  // face e lies on grid lines of dimension e only
    if (fs == st[d]) continue;
    if (st[d]) lo[d] = -1;  // grid-line point between cells q - 1 and q
    else hi[d] = 1;         // centre between grid lines q and q + 1
  }
  double sum = 0.0;
  int cnt = 0;
  for (int c = lo[2]; c <= hi[2]; ++c)
    for (int b = lo[1]; b <= hi[1]; ++b)
      for (int a = lo[0]; a <= hi[0]; ++a) {
        sum += v[g.idx(i + a, j + b, k + c)];
        ++cnt;
      }
  return sum / cnt;
}

// advected value of f at (i, j, k) for a field of extent ext and staggering st
__device__ double advected(const Geo &g, const History &H, const double *f, const int st[3], const int ext[3],
                           int i, int j, int k, double dt) {
  const long long e0 = g.idx(i, j, k);
  const int q[3] = {i, j, k}, n[3] = {g.nx, g.ny, g.nz};
  for (int d = 0; d < g.ndim; ++d)
    if (st[d] && (q[d] == 0 || q[d] == n[d])) return f[e0];  // free-slip wall: shear stress stays
  const double h[3] = {g.dx, g.dy, g.dz};
  const long long step[3] = {1, g.px, g.plane};
  double adv = 0.0;
  for (int e = 0; e < g.ndim; ++e) {
    const double ve = face_mean(g, H.v[e], e, st, i, j, k);
    double D = 0.0;
    if (ve > 0.0 && q[e] >= 1) D = (f[e0] - f[e0 - step[e]]) / h[e];
    else if (ve < 0.0 && q[e] + 1 < ext[e]) D = (f[e0 + step[e]] - f[e0]) / h[e];
    adv += ve * D;
  }
  return f[e0] - dt * adv;
}

__global__ void k_advect(Geo g, History H, const Scal *sc, double *tn0, double *tn1, double *tn2, double *ts0,
                         double *ts1, double *ts2, double *pout) {
  const Pos3 q = pos3(g);
  if (!q.in) return;
  const int i = q.i, j = q.j, k = q.k;
  const long long e = q.e;
  const double dt = sc->dt;
  const bool centre = i < g.nx && j < g.ny && k < g.nz;
  const int sc0[3] = {0, 0, 0}, extc[3] = {g.nx, g.ny, g.nz};
  double *tno[3] = {tn0, tn1, tn2};
  for (int d = 0; d < g.ndim; ++d)
    tno[d][e] = centre ? advected(g, H, H.tn[d], sc0, extc, i, j, k, dt) : H.tn[d][e];
  pout[e] = centre ? advected(g, H, H.p, sc0, extc, i, j, k, dt) : H.p[e];
  double *tso[3] = {ts0, ts1, ts2};
  const int ns = g.ndim == 3 ? 3 : 1;
  for (int c = 0; c < ns; ++c) {
    int st[3], ext[3];
    if (g.ndim == 2) {
      st[0] = 1; st[1] = 1; st[2] = 0;
    } else {
      st[0] = c != 2; st[1] = c != 1; st[2] = c != 0;
    }
    ext[0] = g.nx + st[0]; ext[1] = g.ny + st[1]; ext[2] = g.nz + st[2];
    const bool in = i < ext[0] && j < ext[1] && k < ext[2];
    tso[c][e] = in ? advected(g, H, H.ts[c], st, ext, i, j, k, dt) : H.ts[c][e];
  }
}

}  // namespace


void launch_start_velocity(const Geo &g, const History &H, const double *const dv[3], const Scal *sc,
                           int started, const double L[3], cudaStream_t st) {
  k_start_velocity<<<blocks_for(g.box), kThreads, 0, st>>>(g, H, dv[0], dv[1], dv[2], sc, started, L[0], L[1],
                                                           L[2]);
}

template <typename T>
void launch_rotation_fields(const Geo &g, const History &H, const Scal *sc, T *const rq[3], T *const rd[2],
                            T *yc, cudaStream_t st) {
  k_rotation_fields<T><<<blocks_for(g.box), kThreads, 0, st>>>(g, H, sc, rq[0], rq[1], rq[2], rd[0], rd[1], yc);
}

template <typename T>
void launch_compose(const Geo &g, const double *const v0[3], const T *const u[3], double *const out[3],
                    cudaStream_t st) {
  k_compose<T><<<blocks_for(g.box), kThreads, 0, st>>>(g, v0[0], v0[1], v0[2], u[0], u[1], u[2], out[0], out[1],
                                                       out[2]);
}

template <typename T>
void launch_commit(const Geo &g, const History &H, const double *const Tn64[3], const double *const Ts64[3],
                   const double *const es64[3], const T *const stn[3], const T *const sts[3], const T *stp,
                   const T *s, const Scal *sc, unsigned long long *n_plastic, cudaStream_t st) {
  k_commit<T><<<blocks_for(g.box), kThreads, 0, st>>>(g, H, Tn64[0], Tn64[1], Tn64[2], Ts64[0], Ts64[1], Ts64[2],
                                                      es64[0], es64[1], es64[2], stn[0], stn[1], stn[2], sts[0],
                                                      sts[1], sts[2], stp, s, sc, n_plastic);
}

template <typename Td, typename Ts>
void launch_convert(Td *dst, const Ts *src, long long n, cudaStream_t st) {
  k_convert<Td, Ts><<<blocks_for(n), kThreads, 0, st>>>(dst, src, n);
}

void launch_line_integrals(const Geo &g, const History &H, double *out2, cudaStream_t st) {
  k_line_integrals<<<1, 32, 0, st>>>(g, H, out2);
}

void launch_pack(const double *box, double *dst, int ex, int ey, int ez, int px, int py, cudaStream_t st) {
  long long n = (long long)ex * ey * ez;
  k_pack<<<blocks_for(n), kThreads, 0, st>>>(box, dst, ex, ey, ez, px, py);
}
void launch_unpack(const double *src, double *box, int ex, int ey, int ez, int px, int py, cudaStream_t st) {
  long long n = (long long)ex * ey * ez;
  k_unpack<<<blocks_for(n), kThreads, 0, st>>>(src, box, ex, ey, ez, px, py);
}

void launch_advect(const Geo &g, const History &H, const Scal *sc, double *const tn_out[3], double *const ts_out[3],
                   double *p_out, cudaStream_t st) {
  k_advect<<<blocks_for(g.box), kThreads, 0, st>>>(g, H, sc, tn_out[0], tn_out[1], tn_out[2], ts_out[0], ts_out[1],
                                                   ts_out[2], p_out);
}

template void launch_rotation_fields<float>(const Geo &, const History &, const Scal *, float *const[3],
                                            float *const[2], float *, cudaStream_t);
template void launch_rotation_fields<double>(const Geo &, const History &, const Scal *, double *const[3],
                                             double *const[2], double *, cudaStream_t);
template void launch_compose<float>(const Geo &, const double *const[3], const float *const[3],
                                    double *const[3], cudaStream_t);
template void launch_compose<double>(const Geo &, const double *const[3], const double *const[3],
                                     double *const[3], cudaStream_t);
template void launch_commit<float>(const Geo &, const History &, const double *const[3], const double *const[3],
                                   const double *const[3], const float *const[3], const float *const[3],
                                   const float *, const float *, const Scal *, unsigned long long *, cudaStream_t);
template void launch_commit<double>(const Geo &, const History &, const double *const[3], const double *const[3],
                                    const double *const[3], const double *const[3], const double *const[3],
                                    const double *, const double *, const Scal *, unsigned long long *,
                                    cudaStream_t);
template void launch_convert<float, double>(float *, const double *, long long, cudaStream_t);
template void launch_convert<double, float>(double *, const float *, long long, cudaStream_t);
template void launch_convert<double, double>(double *, const double *, long long, cudaStream_t);

void launch_scaled_div(const Geo &g, const double *const v[3], double scale, double *out, cudaStream_t st) {
  k_scaled_div<<<blocks_for(g.box), kThreads, 0, st>>>(g, v[0], v[1], v[2], scale, out);
}

void launch_shear_fields(const Geo &g, const double *Gc, double mu_s, double dt, double *const ge[4],
                         double *const gc[4], cudaStream_t st) {
  k_shear_fields<<<blocks_for(g.box), kThreads, 0, st>>>(g, Gc, mu_s, dt, ge[0], ge[1], ge[2], ge[3], gc[0], gc[1],
                                                         gc[2], gc[3]);
}

}  // namespace ep
