// ep_warm.cu -- the learned warm start's tensors: features before an
// increment, training targets after it, and the start state built from the
// network's prediction.
//
// The network works on a grid of coarse cells, each the mean of f^D fine
// cells (f = the coarsening factor; 1 keeps the grid), padded with zeros to a
// multiple of 4 cells per side.  Channels, at coarse-cell centres:
//   features (3D: 13, 2D: 9)
//     dv_prev / S_v           (nd)  centre mean of v_{n-1} - v_{n-2}
//     tau_hat_normal / c      (nd)  old deviator at the centre
//     tau_hat_shear / c       (ns)  old shear deviator, mean of the 4 edges
//     p_hat / c               (1)
//     1 - s                   (1)   last return scale of the previous solve
//     c / max c               (1)
//     eps_pl / S_e            (1)
//   targets / outputs (3D: 9, 2D: 5)
//     (v_n - v_{n-1}) / S_v   (nd)  centre mean
//     (tau_n - tau_phys) / S_t (nd + ns)
// with S_v = 0.1 |a| L_max, S_t = 2 G |a| dt and S_e = 10 |a| dt (|a| the
// largest loading rate), c the cell's cohesion.  tau_n is the increment's
// converged pseudo-time stress state (Eqs. A23ssP at pseudo-steady state) and
// tau_phys the physical response of its converged velocity (the start state
// the solve would take at that velocity, R3 reading): the network predicts
// the velocity change and the relaxed-return part of the stress state.
// A start built from a zero prediction is the plain start.
#include <math.h>

#include "ep_internal.cuh"

namespace ep {

namespace {

constexpr int kT = 256;
inline unsigned nb(long long n) { return (unsigned)((n + kT - 1) / kT); }

struct CoarseCell {
  int I, J, K;
  long long t, nv;
  bool in;
};

__device__ __forceinline__ CoarseCell coarse_cell(int Xc, int Yc, int Zc) {
  CoarseCell c;
  c.t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  c.nv = (long long)Xc * Yc * Zc;
  c.in = c.t < c.nv;
  c.I = (int)(c.t % Xc);
  c.J = (int)((c.t / Xc) % Yc);
  c.K = (int)(c.t / ((long long)Xc * Yc));
  return c;
}

// the fine cells of coarse cell (I, J, K) that lie inside the grid
struct FineRange {
  int i0, i1, j0, j1, k0, k1;
  __device__ int count() const { return (i1 - i0) * (j1 - j0) * (k1 - k0); }
};

__device__ __forceinline__ FineRange fine_range(const Geo &g, int f, int I, int J, int K) {
  FineRange r;
  r.i0 = I * f; r.i1 = min(r.i0 + f, g.nx);
  r.j0 = J * f; r.j1 = min(r.j0 + f, g.ny);
  if (g.ndim == 3) { r.k0 = K * f; r.k1 = min(r.k0 + f, g.nz); }
  else { r.k0 = K; r.k1 = K == 0 ? 1 : 0; }
  if (r.i1 < r.i0) r.i1 = r.i0;
  if (r.j1 < r.j0) r.j1 = r.j0;
  if (r.k1 < r.k0) r.k1 = r.k0;
  return r;
}

// mean of shear component c over the 4 vertices/edges around centre e
__device__ __forceinline__ double shear_at_centre(const Geo &g, const double *a, int c, long long e) {
  const long long px = g.px, pl = g.plane;
  if (g.ndim == 2 || c == 0) return 0.25 * (a[e] + a[e + 1] + a[e + px] + a[e + px + 1]);
  if (c == 1) return 0.25 * (a[e] + a[e + 1] + a[e + pl] + a[e + pl + 1]);
  return 0.25 * (a[e] + a[e + px] + a[e + pl] + a[e + pl + px]);
}

template <typename T>
__global__ void k_warm_features(Geo g, History H, const double *vp0, const double *vp1, const double *vp2,
                                const T *s_last, WarmScales ws, int f, float *x, int Xc, int Yc, int Zc) {
  const CoarseCell c = coarse_cell(Xc, Yc, Zc);
  if (!c.in) return;
  const int nd = g.ndim, ns = nd == 3 ? 3 : 1;
  const int nch = warm_in_channels(nd);
  double acc[13];
  for (int q = 0; q < 13; ++q) acc[q] = 0.0;
  const FineRange r = fine_range(g, f, c.I, c.J, c.K);
  const double *vp[3] = {vp0, vp1, vp2};
  const long long off[3] = {1, g.px, g.plane};
  for (int k = r.k0; k < r.k1; ++k)
    for (int j = r.j0; j < r.j1; ++j)
      for (int i = r.i0; i < r.i1; ++i) {
        const long long e = g.idx(i, j, k);
        const double coh = H.coh[e];
        const double ic = coh > 0.0 ? 1.0 / coh : 0.0;
        int q = 0;
        for (int d = 0; d < nd; ++d, ++q)
          acc[q] += 0.5 * ((H.v[d][e] - vp[d][e]) + (H.v[d][e + off[d]] - vp[d][e + off[d]])) * ws.sv_inv;
        for (int d = 0; d < nd; ++d, ++q) acc[q] += H.tn[d][e] * ic;
        for (int s = 0; s < ns; ++s, ++q) acc[q] += shear_at_centre(g, H.ts[s], s, e) * ic;
        acc[q++] += H.p[e] * ic;
        acc[q++] += 1.0 - (double)s_last[e];
        acc[q++] += coh * ws.cmax_inv;
        acc[q++] += H.epl[e] * ws.se_inv;
      }
  const int n = r.count();
  const double inv = n > 0 ? 1.0 / n : 0.0;
  for (int q = 0; q < nch; ++q) x[q * c.nv + c.t] = (float)(acc[q] * inv);
}

__global__ void k_warm_target(Geo g, History H, const double *vp0, const double *vp1, const double *vp2,
                              const float *w0, WarmScales ws, int f, float *out, int Xc, int Yc, int Zc) {
  const CoarseCell c = coarse_cell(Xc, Yc, Zc);
  if (!c.in) return;
  const int nd = g.ndim, ns = nd == 3 ? 3 : 1;
  const int nch = warm_out_channels(nd);
  double acc[9];
  for (int q = 0; q < 9; ++q) acc[q] = 0.0;
  const FineRange r = fine_range(g, f, c.I, c.J, c.K);
  const double *vp[3] = {vp0, vp1, vp2};
  const long long off[3] = {1, g.px, g.plane};
  const long long px = g.px, pl = g.plane, box = g.box;
  for (int k = r.k0; k < r.k1; ++k)
    for (int j = r.j0; j < r.j1; ++j)
      for (int i = r.i0; i < r.i1; ++i) {
        const long long e = g.idx(i, j, k);
        int q = 0;
        for (int d = 0; d < nd; ++d, ++q)
          acc[q] += 0.5 * ((H.v[d][e] - vp[d][e]) + (H.v[d][e + off[d]] - vp[d][e + off[d]])) * ws.sv_inv;
        for (int d = 0; d < nd; ++d, ++q) acc[q] += (H.tn[d][e] - (double)w0[d * box + e]) * ws.st_inv;
        for (int s = 0; s < ns; ++s, ++q) {
          const double *a = H.ts[s];
          const float *b = w0 + (nd + s) * box;
          long long o1, o2;   // the other three points of the centre's edge ring
          if (nd == 2 || s == 0) { o1 = 1; o2 = px; }
          else if (s == 1) { o1 = 1; o2 = pl; }
          else { o1 = px; o2 = pl; }
          const double m = 0.25 * ((a[e] - (double)b[e]) + (a[e + o1] - (double)b[e + o1]) +
                                   (a[e + o2] - (double)b[e + o2]) + (a[e + o1 + o2] - (double)b[e + o1 + o2]));
          acc[q] += m * ws.st_inv;
        }
      }
  const int n = r.count();
  const double inv = n > 0 ? 1.0 / n : 0.0;
  for (int q = 0; q < nch; ++q) out[q * c.nv + c.t] = (float)(acc[q] * inv);
}

// w0 <- (tau_phys normal components, tau_phys shear components), FP32 boxes
__global__ void k_warm_record(Geo g, const double *n0, const double *n1, const double *n2, const double *s0,
                              const double *s1, const double *s2, float *w0) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.box) return;
  const int nd = g.ndim;
  const double *src[6] = {n0, n1, n2, s0, s1, s2};
  int q = 0;
  for (int d = 0; d < nd; ++d, ++q) w0[q * g.box + e] = (float)src[d][e];
  for (int s = 0; s < (nd == 3 ? 3 : 1); ++s, ++q) w0[q * g.box + e] = (float)src[3 + s][e];
}

// the network's channel q at a fine position (px_, py_, pz_ in fine-cell
// units, cell i spanning [i, i+1)), interpolated linearly between the
// coarse-cell centres around it (clamped to the coarse cells that cover the
// grid)
__device__ __forceinline__ double interp(const float *y, int q, long long nv, int Xc, int Yc, int ncx, int ncy,
                                         int ncz, int f, int nd, double fx, double fy, double fz) {
  const double inv = 1.0 / f;
  double cx = fx * inv - 0.5, cy = fy * inv - 0.5, cz = nd == 3 ? fz * inv - 0.5 : 0.0;
  cx = fmin(fmax(cx, 0.0), (double)(ncx - 1));
  cy = fmin(fmax(cy, 0.0), (double)(ncy - 1));
  cz = fmin(fmax(cz, 0.0), (double)(ncz - 1));
  const int x0 = min((int)cx, ncx - 1), y0 = min((int)cy, ncy - 1), z0 = min((int)cz, ncz - 1);
  const int x1 = min(x0 + 1, ncx - 1), y1 = min(y0 + 1, ncy - 1), z1 = min(z0 + 1, ncz - 1);
  const double ax = cx - x0, ay = cy - y0, az = cz - z0;
  const float *b = y + q * nv;
  auto at = [&](int X, int Y, int Z) { return (double)b[((long long)Z * Yc + Y) * Xc + X]; };
  const double v00 = (1 - ax) * at(x0, y0, z0) + ax * at(x1, y0, z0);
  const double v10 = (1 - ax) * at(x0, y1, z0) + ax * at(x1, y1, z0);
  const double v01 = (1 - ax) * at(x0, y0, z1) + ax * at(x1, y0, z1);
  const double v11 = (1 - ax) * at(x0, y1, z1) + ax * at(x1, y1, z1);
  return (1 - az) * ((1 - ay) * v00 + ay * v10) + az * ((1 - ay) * v01 + ay * v11);
}

// start increment at interior faces from the velocity channels
__global__ void k_warm_dv(Geo g, const float *y, int f, double sv, double *dv0, double *dv1, double *dv2, int Xc,
                          int Yc, int Zc) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.box) return;
  const int i = (int)(e % g.px), j = (int)((e / g.px) % g.py), k = (int)(e / g.plane);
  const int nd = g.ndim, ez = nd == 3 ? g.nz : 1;
  const long long nv = (long long)Xc * Yc * Zc;
  const int ncx = (g.nx + f - 1) / f, ncy = (g.ny + f - 1) / f, ncz = nd == 3 ? (g.nz + f - 1) / f : 1;
  double *dv[3] = {dv0, dv1, dv2};
  for (int d = 0; d < nd; ++d) {
    const int ext[3] = {g.nx + (d == 0), g.ny + (d == 1), ez + (d == 2)};
    const int idx3[3] = {i, j, k};
    const bool in = i < ext[0] && j < ext[1] && k < ext[2];
    const bool wall = idx3[d] == 0 || idx3[d] == (d == 0 ? g.nx : d == 1 ? g.ny : g.nz);
    double v = 0.0;
    if (in && !wall) {
      const double fx = d == 0 ? i : i + 0.5, fy = d == 1 ? j : j + 0.5, fz = d == 2 ? k : k + 0.5;
      v = sv * interp(y, d, nv, Xc, Yc, ncx, ncy, ncz, f, nd, fx, fy, fz);
    }
    dv[d][e] = v;
  }
}

// add the stress channels to a start state (centres and interior edges)
__global__ void k_warm_stress(Geo g, const float *y, int f, double st, double *n0, double *n1, double *n2,
                              double *s0, double *s1, double *s2, int Xc, int Yc, int Zc) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.box) return;
  const int i = (int)(e % g.px), j = (int)((e / g.px) % g.py), k = (int)(e / g.plane);
  const int nd = g.ndim, ns = nd == 3 ? 3 : 1, ez = nd == 3 ? g.nz : 1;
  const long long nv = (long long)Xc * Yc * Zc;
  const int ncx = (g.nx + f - 1) / f, ncy = (g.ny + f - 1) / f, ncz = nd == 3 ? (g.nz + f - 1) / f : 1;
  double *nn[3] = {n0, n1, n2}, *ss[3] = {s0, s1, s2};
  if (i < g.nx && j < g.ny && k < ez)
    for (int d = 0; d < nd; ++d)
      nn[d][e] += st * interp(y, nd + d, nv, Xc, Yc, ncx, ncy, ncz, f, nd, i + 0.5, j + 0.5, k + 0.5);
  for (int s = 0; s < ns; ++s) {
    // shear points: 2D vertices / 3D xy-edges on x and y lines, xz on x and
    // z lines, yz on y and z lines; the wall ones stay zero (free slip)
    const bool on_x = nd == 2 || s != 2, on_y = nd == 2 || s != 1, on_z = nd == 3 && s != 0;
    const bool ix = on_x ? (i >= 1 && i <= g.nx - 1) : i < g.nx;
    const bool jy = on_y ? (j >= 1 && j <= g.ny - 1) : j < g.ny;
    const bool kz = on_z ? (k >= 1 && k <= g.nz - 1) : k < ez;
    if (!(ix && jy && kz)) continue;
    ss[s][e] += st * interp(y, 2 * nd + s, nv, Xc, Yc, ncx, ncy, ncz, f, nd, on_x ? i : i + 0.5,
                            on_y ? j : j + 0.5, on_z ? k : k + 0.5);
  }
}

}  // namespace

template <typename T>
void launch_warm_features(const Geo &g, const History &H, const double *const vp[3], const T *s_last,
                          const WarmScales &ws, int f, float *x, const int dims[3], cudaStream_t st) {
  const long long nv = (long long)dims[0] * dims[1] * dims[2];
  k_warm_features<T><<<nb(nv), kT, 0, st>>>(g, H, vp[0], vp[1], vp[2], s_last, ws, f, x, dims[0], dims[1], dims[2]);
}
template void launch_warm_features<float>(const Geo &, const History &, const double *const[3], const float *,
                                          const WarmScales &, int, float *, const int[3], cudaStream_t);
template void launch_warm_features<double>(const Geo &, const History &, const double *const[3], const double *,
                                           const WarmScales &, int, float *, const int[3], cudaStream_t);

void launch_warm_target(const Geo &g, const History &H, const double *const vp[3], const float *w0,
                        const WarmScales &ws, int f, float *out, const int dims[3], cudaStream_t st) {
  const long long nv = (long long)dims[0] * dims[1] * dims[2];
  k_warm_target<<<nb(nv), kT, 0, st>>>(g, H, vp[0], vp[1], vp[2], w0, ws, f, out, dims[0], dims[1], dims[2]);
}

void launch_warm_record(const Geo &g, const double *const n[3], const double *const s[3], float *w0,
                        cudaStream_t st) {
  k_warm_record<<<nb(g.box), kT, 0, st>>>(g, n[0], n[1], n[2], s[0], s[1], s[2], w0);
}

void launch_warm_dv(const Geo &g, const float *y, int f, double sv, double *const dv[3], const int dims[3],
                    cudaStream_t st) {
  k_warm_dv<<<nb(g.box), kT, 0, st>>>(g, y, f, sv, dv[0], dv[1], dv[2], dims[0], dims[1], dims[2]);
}

void launch_warm_stress(const Geo &g, const float *y, int f, double stress_scale, double *const n[3],
                        double *const s[3], const int dims[3], cudaStream_t st) {
  k_warm_stress<<<nb(g.box), kT, 0, st>>>(g, y, f, stress_scale, n[0], n[1], n[2], s[0], s[1], s[2], dims[0],
                                          dims[1], dims[2]);
}

}  // namespace ep
