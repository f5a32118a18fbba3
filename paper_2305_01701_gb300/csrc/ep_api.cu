// ep_api.cu -- host side of libep: handles, the device arena, the
// per-increment prologue, the graph-captured iteration loop and the commit.
//
// Memory plan (one arena per grid, every array a full padded box):
//   FP64 history ........ converged v, old deviator, p, cohesion, plastic
//                         strain, displacement, accumulated strain, start v
//   FP64 scratch ........ physical response at the start / converged velocity
//   sweep state (T) ..... velocity increment u and stress state, ping-pong
//   sweep constants (T) . base trial, base pressure, B c, rotation weights
// The sweep of one load increment runs as chunks of n_chk iterations, each
// chunk one CUDA graph (5 stage kernels per iteration plus one check kernel);
// the host reads a 100-byte status once per chunk.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ep_internal.cuh"

using namespace ep;

struct ep_grid {
  int ndim = 2, n[3] = {1, 1, 1};
  double L[3] = {1, 1, 1};
  Geo g{};
  ep_precision prec = EP_FP64;
  cudaStream_t stream = nullptr, cap = nullptr;
  bool own_stream = false;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  bool own_arena = false;
  double K = 0, G = 0, mu_s = 0, A = 0, B = 0;
  bool have_material = false;
  ep_solver_opts opts{};
  double rate[3] = {0, 0, 0}, dt = 0;
  bool in_increment = false, started = false, have_f = false;
  bool solving = false;          // a solve of the open increment is under way (ep_solve_chunks)
  History H{};
  // FP64 scratch
  double *om64[3] = {}, *es64[3] = {}, *Tn64[3] = {}, *Ts64[3] = {}, *s64 = nullptr;
  double *stn64[3] = {}, *sts64[3] = {}, *stp64 = nullptr, *rq64[3] = {}, *rd64[2] = {}, *yc64 = nullptr;
  double *stage64 = nullptr;  // host-transfer staging (one box)
  // sweep arrays (element type T = double or float)
  void *u[2][3] = {}, *stn[2][3] = {}, *sts[2][3] = {}, *stp[2] = {};
  void *tbn[3] = {}, *tbs[3] = {}, *pb = nullptr, *yc = nullptr, *rq[3] = {}, *rd[2] = {};
  void *om[3] = {}, *es[3] = {}, *Tn[3] = {}, *Ts[3] = {}, *s = nullptr, *uchk[3] = {}, *f[3] = {};
  void *cn[3] = {}, *cs[3] = {}, *cp = nullptr;  // stress state at the previous check
  // small device / pinned blocks
  Scal *dscal = nullptr;
  DevInfo *dinfo = nullptr, *hinfo = nullptr;
  unsigned long long *dnpl = nullptr;
  double *dline = nullptr;
  cudaGraphExec_t chunk = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int variant = EP_KERNEL_AUTO;  // sweep kernel choice (ep_set_kernel)
  int kz = 0;               // z-planes per CTA of the fused 3D kernel (0: by grid size)
  int tile = 0;             // tile of the fused 2D kernel (0: 32x8, 1: 32x16, 2: 64x8)
  void *inst_dev = nullptr; // this grid as a batch of one (fused 2D)
  int4 *items_dev = nullptr;
  int n_items = 0, items_tile = -1, max_items = 0;
  double last_rate[3] = {0, 0, 0};
  // learned warm start
  double *vpp[3] = {};          // converged velocity of the increment before last
  int n_commits = 0;
  int adv_done = 0;             // n_commits when the history was last advected
  double cmax = 1.0;
  ep_net *net = nullptr;
  float *wx = nullptr, *wy = nullptr;   // network input / output (cudaMalloc on attach)
  int wcoarse = 1;              // coarsening factor of the attached network's grid
  bool warm_stress = false;     // the next prologue adds the predicted stress state
  bool wrecord = false;         // commits record the physical response (training targets)
  float *w0 = nullptr;          // that response, (nd + ns) FP32 boxes (cudaMalloc)
  // per-cell shear modulus (ep_set_shear_modulus; cudaMalloc, null: uniform G)
  double *Gc = nullptr;         // at centres
  double Gmax = 0.0;
  double *ge64[4] = {}, *gc64[4] = {};   // 2 eta_ve and c2 at centres and vertices/edges
  void *geT[4] = {}, *gcT[4] = {};       // their sweep-type copies
  char *snap = nullptr;     // checkpoint of the history (ep_snapshot)
  bool snap_started = false;
  int snap_commits = 0, snap_adv_done = 0;
  std::string err;
};

static thread_local std::string g_thread_err;

static ep_status fail(ep_grid *h, ep_status st, const std::string &msg) {
  if (h) h->err = msg;
  g_thread_err = msg;
  return st;
}

#define CK(h, call)                                                                                 \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      return fail((h), e_ == cudaErrorMemoryAllocation ? EP_ERR_OOM : EP_ERR_CUDA,                  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                               \
    }                                                                                               \
  } while (0)

namespace {

int n_shear(int ndim) { return ndim == 3 ? 3 : 1; }

struct Arena {
  char *base = nullptr;
  size_t off = 0;
  bool dry = true;
  template <typename T>
  T *take(long long n) {
    size_t b = ((size_t)n * sizeof(T) + 255) & ~(size_t)255;
    T *p = dry ? nullptr : (T *)(base + off);
    off += b;
    return p;
  }
};

Geo make_geo(int ndim, const int n[3], const double L[3]) {
  Geo g{};
  g.ndim = ndim;
  g.nx = n[0];
  g.ny = n[1];
  g.nz = ndim == 3 ? n[2] : 1;
  g.px = ((g.nx + 1) + 31) / 32 * 32;
  g.py = g.ny + 1;
  g.pz = ndim == 3 ? g.nz + 1 : 1;
  g.plane = (long long)g.px * g.py;
  g.box = g.plane * g.pz;
  g.dx = L[0] / g.nx;
  g.dy = L[1] / g.ny;
  g.dz = ndim == 3 ? L[2] / g.nz : 1.0;
  g.rdx = 1.0 / g.dx;
  g.rdy = 1.0 / g.dy;
  g.rdz = 1.0 / g.dz;
  return g;
}

// Assign every array of h from the arena (dry run: only count bytes).
void carve(ep_grid *h, Arena &a) {
  const long long B = h->g.box;
  const int nd = h->ndim, ns = n_shear(nd);
  const size_t es = h->prec == EP_FP64 ? sizeof(double) : sizeof(float);
  auto tk = [&](void *&p) {
    if (es == 8) p = a.take<double>(B); else p = a.take<float>(B);
  };
  for (int d = 0; d < nd; ++d) {
    h->vpp[d] = a.take<double>(B);
    h->H.v[d] = a.take<double>(B); h->H.u[d] = a.take<double>(B); h->H.v0[d] = a.take<double>(B);
    h->H.tn[d] = a.take<double>(B); h->H.an[d] = a.take<double>(B);
    h->Tn64[d] = a.take<double>(B); h->stn64[d] = a.take<double>(B);
  }
  for (int c = 0; c < ns; ++c) {
    h->H.ts[c] = a.take<double>(B); h->H.as[c] = a.take<double>(B);
    h->om64[c] = a.take<double>(B); h->es64[c] = a.take<double>(B); h->Ts64[c] = a.take<double>(B);
    h->sts64[c] = a.take<double>(B); h->rq64[c] = a.take<double>(B);
  }
  h->H.p = a.take<double>(B); h->H.coh = a.take<double>(B); h->H.epl = a.take<double>(B);
  h->s64 = a.take<double>(B); h->stp64 = a.take<double>(B); h->yc64 = a.take<double>(B);
  h->rd64[0] = a.take<double>(B);
  if (nd == 3) h->rd64[1] = a.take<double>(B);
  h->stage64 = a.take<double>(B);
  for (int b = 0; b < 2; ++b) {
    for (int d = 0; d < nd; ++d) { tk(h->u[b][d]); tk(h->stn[b][d]); }
    for (int c = 0; c < ns; ++c) tk(h->sts[b][c]);
    tk(h->stp[b]);
  }
  for (int d = 0; d < nd; ++d) { tk(h->tbn[d]); tk(h->Tn[d]); tk(h->uchk[d]); tk(h->f[d]); tk(h->cn[d]); }
  for (int c = 0; c < ns; ++c) {
    tk(h->tbs[c]); tk(h->rq[c]); tk(h->om[c]); tk(h->es[c]); tk(h->Ts[c]); tk(h->cs[c]);
  }
  tk(h->pb); tk(h->yc); tk(h->s); tk(h->rd[0]); tk(h->cp);
  if (nd == 3) tk(h->rd[1]);
  h->dscal = a.take<Scal>(1);
  h->dinfo = a.take<DevInfo>(1);
  h->inst_dev = a.take<Inst2<double>>(1);
  h->max_items = ((h->g.px + 31) / 32) * ((h->g.py + 7) / 8);
  h->items_dev = a.take<int4>(h->max_items);
  h->dnpl = a.take<unsigned long long>(1);
  h->dline = a.take<double>(2);
}

// natural extent of a field id; returns false for an unknown / absent field
bool field_extent(const ep_grid *h, int f, int &ex, int &ey, int &ez) {
  const int nx = h->g.nx, ny = h->g.ny, nz = h->g.nz, nd = h->ndim;
  auto face = [&](int d) {
    ex = nx + (d == 0); ey = ny + (d == 1); ez = nz + (d == 2);
    return d < nd;
  };
  switch (f) {
    case EP_VX: case EP_UX: case EP_V0X: return face(0);
    case EP_VY: case EP_UY: case EP_V0Y: return face(1);
    case EP_VZ: case EP_UZ: case EP_V0Z: return face(2);
    case EP_TXX: case EP_TYY: case EP_P: case EP_EPL: case EP_EXX: case EP_EYY: case EP_COH: case EP_EII:
    case EP_SCALE:
      ex = nx; ey = ny; ez = nz; return true;
    case EP_TZZ: case EP_EZZ: ex = nx; ey = ny; ez = nz; return nd == 3;
    case EP_TXY: case EP_EXY: ex = nx + 1; ey = ny + 1; ez = nz; return true;
    case EP_TXZ: case EP_EXZ: ex = nx + 1; ey = ny; ez = nz + 1; return nd == 3;
    case EP_TYZ: case EP_EYZ: ex = nx; ey = ny + 1; ez = nz + 1; return nd == 3;
    default: return false;
  }
}

double *history_ptr(ep_grid *h, int f) {
  switch (f) {
    case EP_VX: return h->H.v[0]; case EP_VY: return h->H.v[1]; case EP_VZ: return h->H.v[2];
    case EP_TXX: return h->H.tn[0]; case EP_TYY: return h->H.tn[1]; case EP_TZZ: return h->H.tn[2];
    case EP_TXY: return h->H.ts[0]; case EP_TXZ: return h->H.ts[1]; case EP_TYZ: return h->H.ts[2];
    case EP_P: return h->H.p; case EP_EPL: return h->H.epl; case EP_COH: return h->H.coh;
    case EP_UX: return h->H.u[0]; case EP_UY: return h->H.u[1]; case EP_UZ: return h->H.u[2];
    case EP_EXX: return h->H.an[0]; case EP_EYY: return h->H.an[1]; case EP_EZZ: return h->H.an[2];
    case EP_EXY: return h->H.as[0]; case EP_EXZ: return h->H.as[1]; case EP_EYZ: return h->H.as[2];
    case EP_V0X: return h->H.v0[0]; case EP_V0Y: return h->H.v0[1]; case EP_V0Z: return h->H.v0[2];
    default: return nullptr;
  }
}

// host -> padded device box (via the FP64 staging buffer)
ep_status upload_box(ep_grid *h, const double *host, double *box, int ex, int ey, int ez) {
  size_t n = (size_t)ex * ey * ez;
  CK(h, cudaMemcpyAsync(h->stage64, host, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  launch_unpack(h->stage64, box, ex, ey, ez, h->g.px, h->g.py, h->stream);
  CK(h, cudaGetLastError());
  CK(h, cudaStreamSynchronize(h->stream));
  return EP_OK;
}

ep_status download_box(ep_grid *h, const double *box, double *host, int ex, int ey, int ez) {
  size_t n = (size_t)ex * ey * ez;
  launch_pack(box, h->stage64, ex, ey, ez, h->g.px, h->g.py, h->stream);
  CK(h, cudaGetLastError());
  CK(h, cudaMemcpyAsync(host, h->stage64, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return EP_OK;
}

double eta_ve(const ep_grid *h) {
  return isinf(h->mu_s) ? h->G * h->dt : 1.0 / (1.0 / (h->G * h->dt) + 1.0 / h->mu_s);
}

// Numerical parameters of Eqs. PT1-PT24qq with pseudo-time step 1:
// Vp = C dx_min, rho~ = Re eta_ve / (Vp L_max), G~ = rho~ Vp^2 / (r + 4/3),
// K~ = r G~, Re = xi 3 sqrt(10) pi / 2.
Scal make_scal(const ep_grid *h) {
  Scal s{};
  // the pseudo-transient parameters take the largest modulus of a per-cell G
  const double eta = h->Gc ? (isinf(h->mu_s) ? h->Gmax * h->dt : 1.0 / (1.0 / (h->Gmax * h->dt) + 1.0 / h->mu_s))
                           : eta_ve(h);
  s.gcell = h->Gc != nullptr;
  s.two_eta = 2.0 * eta;
  s.c2 = eta / (h->G * h->dt);
  s.c2dt = s.c2 * h->dt;
  s.KDt = h->K * h->dt;
  s.A = h->A;
  s.B = h->B;
  s.dt = h->dt;
  s.tol = h->opts.tol;
  s.n_chk = h->opts.n_chk;
  s.jaumann = h->opts.jaumann;
  // frozen plasticity: the paper's rule (16 n_x on grids above 10^6 cells)
  // unless the caller set freeze_iter
  long long fi = h->opts.freeze_iter;
  if (fi < 0) fi = (double)h->g.nx * h->g.ny * h->g.nz > 1e6 ? 16LL * h->g.nx : 0;
  s.freeze_iter = fi;
  s.freeze_eps = h->opts.freeze_eps;
  s.wait_cycles = h->opts.wait_cycles;
  double dxm = std::min(h->g.dx, h->g.dy), Lm = std::max(h->L[0], h->L[1]);
  if (h->ndim == 3) { dxm = std::min(dxm, h->g.dz); Lm = std::max(Lm, h->L[2]); }
  s.dxmin = dxm;
  const double Re = h->opts.xi * 3.0 * sqrt(10.0) * M_PI / 2.0, r = h->opts.r_pt;
  const double Vp = h->opts.c_cfl * dxm;
  const double rho = Re * eta / (Vp * Lm);
  const double Gt = rho * Vp * Vp / (r + 4.0 / 3.0);
  const double Kt = r * Gt;
  s.bt = (1.0 / (2.0 * Gt)) / (1.0 / (2.0 * Gt) + 1.0 / (2.0 * eta));
  s.bp = (1.0 / Kt) / (1.0 / Kt + 1.0 / (h->K * h->dt));
  s.vstep = 1.0 / rho;
  s.inv_1mbt = 1.0 / (1.0 - s.bt);
  s.inv_1mbp = 1.0 / (1.0 - s.bp);
  if (h->opts.incompressible) {
    // Eq. A2ssP2 with pseudo step 1: p_{k+1} = p_k - K~ div v; the pressure
    // is no function of v, so the physical response keeps p_hat, and its
    // measure is 2 eta_ve <|div v|> (reading R9)
    s.bp = 1.0;
    s.obp = 1.0;
    s.KDt = Kt;
    s.KDt_phys = 0.0;
    s.p_meas = 2.0 * eta / Kt;
  } else {
    s.obp = 1.0 - s.bp;
    s.KDt_phys = s.KDt;
    s.p_meas = s.inv_1mbp;
  }
  for (int d = 0; d < 3; ++d) s.rate[d] = h->rate[d];
  return s;
}

template <typename T>
T *P(void *p) { return (T *)p; }

// Stage of sweep iteration parity b: reads buffer b, writes buffer 1 - b.
template <typename T>
Stage<T> sweep_stage(ep_grid *h, int b) {
  Stage<T> S{};
  const int o = 1 - b;
  for (int d = 0; d < 3; ++d) {
    S.u[d] = P<T>(h->u[b][d]); S.uo[d] = P<T>(h->u[o][d]);
    S.son[d] = P<T>(h->stn[b][d]); S.snn[d] = P<T>(h->stn[o][d]);
    S.sos[d] = P<T>(h->sts[b][d]); S.sns[d] = P<T>(h->sts[o][d]);
    S.tbn[d] = P<T>(h->tbn[d]); S.tbs[d] = P<T>(h->tbs[d]); S.rq[d] = P<T>(h->rq[d]);
    S.om[d] = P<T>(h->om[d]); S.es[d] = P<T>(h->es[d]); S.Tn[d] = P<T>(h->Tn[d]); S.Ts[d] = P<T>(h->Ts[d]);
    S.uchk[d] = P<T>(h->uchk[d]); S.v0[d] = h->H.v0[d];
    S.cn[d] = P<T>(h->cn[d]); S.cs[d] = P<T>(h->cs[d]);
    S.f[d] = h->have_f ? P<T>(h->f[d]) : nullptr;
  }
  S.sop = P<T>(h->stp[b]); S.snp = P<T>(h->stp[o]); S.cp = P<T>(h->cp);
  S.pb = P<T>(h->pb); S.yc = P<T>(h->yc); S.s = P<T>(h->s);
  S.rd[0] = P<T>(h->rd[0]); S.rd[1] = P<T>(h->rd[1]);
  S.tb_scale = 1.0;
  S.tb_c2 = 0;
  S.relax = 1;
  for (int w = 0; w < 4; ++w) {
    S.ge[w] = h->Gc ? P<T>(h->geT[w]) : nullptr;
    S.gc[w] = h->Gc ? P<T>(h->gcT[w]) : nullptr;
  }
  return S;
}

// This grid as one instance of the batched fused 2D kernel.
template <typename T>
Inst2<T> make_inst(ep_grid *h, DevInfo *di) {
  Inst2<T> I{};
  I.g = h->g;
  I.sc = h->dscal;
  I.di = di;
  for (int b = 0; b < 2; ++b) {
    for (int d = 0; d < 2; ++d) { I.u[b][d] = P<T>(h->u[b][d]); I.sn[b][d] = P<T>(h->stn[b][d]); }
    I.ss[b] = P<T>(h->sts[b][0]);
    I.sp[b] = P<T>(h->stp[b]);
  }
  for (int d = 0; d < 2; ++d) {
    I.tbn[d] = P<T>(h->tbn[d]); I.uchk[d] = P<T>(h->uchk[d]); I.cn[d] = P<T>(h->cn[d]); I.v0[d] = h->H.v0[d];
  }
  I.tbs = P<T>(h->tbs[0]); I.pb = P<T>(h->pb); I.yc = P<T>(h->yc); I.rq = P<T>(h->rq[0]); I.rd = P<T>(h->rd[0]);
  I.s = P<T>(h->s); I.cs = P<T>(h->cs[0]); I.cp = P<T>(h->cp);
  return I;
}

// (instance, tile_x, tile_y) work items covering the padded box of a grid
void append_items(std::vector<int4> &v, int inst, const Geo &g, int tile) {
  int tx, ty;
  fused2d_tile(tile, &tx, &ty);
  for (int j = 0; j < (g.py + ty - 1) / ty; ++j)
    for (int i = 0; i < (g.px + tx - 1) / tx; ++i) v.push_back(make_int4(inst, i, j, 0));
}

template <typename T>
bool use_fused2d(const ep_grid *h) {
  if (h->ndim != 2 || h->have_f || h->Gc) return false;
  return h->variant == EP_KERNEL_FUSED || (h->variant == EP_KERNEL_AUTO && sizeof(T) == 4);
}

// upload this grid's instance record and work items for its tile
template <typename T>
ep_status prepare_solo2d(ep_grid *h) {
  Inst2<T> I = make_inst<T>(h, h->dinfo);
  CK(h, cudaMemcpyAsync(h->inst_dev, &I, sizeof(I), cudaMemcpyHostToDevice, h->stream));
  if (h->items_tile != h->tile) {
    std::vector<int4> it;
    append_items(it, 0, h->g, h->tile);
    if ((int)it.size() > h->max_items) return fail(h, EP_ERR_ARG, "work-item list larger than reserved");
    CK(h, cudaMemcpyAsync(h->items_dev, it.data(), it.size() * sizeof(int4), cudaMemcpyHostToDevice, h->stream));
    h->n_items = (int)it.size();
    h->items_tile = h->tile;
  }
  CK(h, cudaStreamSynchronize(h->stream));
  return EP_OK;
}

int persistent_blocks(int tile, size_t elem) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per = elem == 4 ? fused2d_blocks_per_sm<float>(tile) : fused2d_blocks_per_sm<double>(tile);
  return sms * per;
}

// FP64 physical response at face field v (beta = 0, base = c2 tau_hat).
Stage<double> phys_stage(ep_grid *h, double *const v[3]) {
  Stage<double> S{};
  for (int d = 0; d < 3; ++d) {
    S.u[d] = v[d];
    S.snn[d] = h->stn64[d]; S.sns[d] = h->sts64[d];
    S.tbn[d] = h->H.tn[d]; S.tbs[d] = h->H.ts[d]; S.rq[d] = h->rq64[d];
    S.om[d] = h->om64[d]; S.es[d] = h->es64[d]; S.Tn[d] = h->Tn64[d]; S.Ts[d] = h->Ts64[d];
  }
  S.snp = h->stp64; S.pb = h->H.p; S.yc = h->yc64; S.s = h->s64;
  S.rd[0] = h->rd64[0]; S.rd[1] = h->rd64[1];
  S.tb_scale = make_scal(h).c2;
  S.tb_c2 = 1;
  S.relax = 0;
  for (int w = 0; w < 4; ++w) {
    S.ge[w] = h->Gc ? h->ge64[w] : nullptr;
    S.gc[w] = h->Gc ? h->gc64[w] : nullptr;
  }
  return S;
}

// padded size of the warm-start network's grid at coarsening f
void warm_dims(const ep_grid *h, int f, int dims[3]) {
  dims[0] = ((h->g.nx + f - 1) / f + 3) / 4 * 4;
  dims[1] = ((h->g.ny + f - 1) / f + 3) / 4 * 4;
  dims[2] = h->ndim == 3 ? ((h->g.nz + f - 1) / f + 3) / 4 * 4 : 1;
}

WarmScales warm_scales(const ep_grid *h) {
  double a = 0.0, Lm = 0.0;
  for (int d = 0; d < h->ndim; ++d) { a = std::max(a, fabs(h->rate[d])); Lm = std::max(Lm, h->L[d]); }
  if (!(a > 0.0)) a = 1.0;
  const double dt = h->dt > 0.0 ? h->dt : 1.0;
  WarmScales w;
  w.sv_inv = 1.0 / (0.1 * a * Lm);
  w.st_inv = 1.0 / (2.0 * h->G * a * dt);
  w.se_inv = 1.0 / (10.0 * a * dt);
  w.cmax_inv = 1.0 / h->cmax;
  return w;
}

template <typename Td>
ep_status copy_into(ep_grid *h, void *dst, const double *src) {
  if (sizeof(Td) == 8) {
    CK(h, cudaMemcpyAsync(dst, src, h->g.box * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  } else {
    launch_convert<float, double>((float *)dst, src, h->g.box, h->stream);
  }
  return EP_OK;
}

// Start of an increment: start velocity, rotation weights, the physical
// response at the start velocity (the first pseudo-time state) and the sweep
// constants, all from FP64.
template <typename T>
ep_status prologue(ep_grid *h, const double *const dv[3]) {
  const Geo &g = h->g;
  cudaStream_t st = h->stream;
  launch_start_velocity(g, h->H, dv, h->dscal, h->started ? 1 : 0, h->L, st);
  if (h->opts.advection && h->n_commits > h->adv_done) {
    // transport the old stress with the last converged velocity H.v (Eq. j1);
    // Tn64 / Ts64 / stp64 are free here (dv was consumed above)
    const int nd = h->ndim, ns = n_shear(nd);
    launch_advect(g, h->H, h->dscal, h->Tn64, h->Ts64, h->stp64, st);
    for (int d = 0; d < nd; ++d)
      CK(h, cudaMemcpyAsync(h->H.tn[d], h->Tn64[d], g.box * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (int c = 0; c < ns; ++c)
      CK(h, cudaMemcpyAsync(h->H.ts[c], h->Ts64[c], g.box * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(h, cudaMemcpyAsync(h->H.p, h->stp64, g.box * sizeof(double), cudaMemcpyDeviceToDevice, st));
    h->adv_done = h->n_commits;
  }
  launch_rotation_fields<double>(g, h->H, h->dscal, h->rq64, h->rd64, h->yc64, st);
  Stage<double> S = phys_stage(h, h->H.v0);
  launch_strain<double>(g, S, h->dscal, nullptr, st);
  launch_trial<double>(g, S, h->dscal, nullptr, st);
  launch_return_centres<double>(g, S, h->dscal, nullptr, 0, st);
  launch_return_edges<double>(g, S, h->dscal, nullptr, 0, st);
  if (h->warm_stress && h->net) {
    // learned warm start: the predicted relaxed-return part of the state
    int dims[3];
    warm_dims(h, h->wcoarse, dims);
    launch_warm_stress(g, h->wy, h->wcoarse, 1.0 / warm_scales(h).st_inv, h->stn64, h->sts64, dims, st);
  }
  CK(h, cudaGetLastError());
  // sweep constants: base trial tau_tr(v0), base pressure p(v0), weights
  const int nd = h->ndim, ns = n_shear(nd);
  for (int d = 0; d < nd; ++d) {
    if (copy_into<T>(h, h->tbn[d], h->Tn64[d]) != EP_OK) return EP_ERR_CUDA;
    if (copy_into<T>(h, h->stn[0][d], h->stn64[d]) != EP_OK) return EP_ERR_CUDA;
    if (copy_into<T>(h, h->stn[1][d], h->stn64[d]) != EP_OK) return EP_ERR_CUDA;
    if (copy_into<T>(h, h->cn[d], h->stn64[d]) != EP_OK) return EP_ERR_CUDA;
    CK(h, cudaMemsetAsync(h->u[0][d], 0, g.box * sizeof(T), st));
    CK(h, cudaMemsetAsync(h->u[1][d], 0, g.box * sizeof(T), st));
    CK(h, cudaMemsetAsync(h->uchk[d], 0, g.box * sizeof(T), st));
  }
  for (int c = 0; c < ns; ++c) {
    if (copy_into<T>(h, h->tbs[c], h->Ts64[c]) != EP_OK) return EP_ERR_CUDA;
    if (copy_into<T>(h, h->sts[0][c], h->sts64[c]) != EP_OK) return EP_ERR_CUDA;
    if (copy_into<T>(h, h->sts[1][c], h->sts64[c]) != EP_OK) return EP_ERR_CUDA;
    if (copy_into<T>(h, h->cs[c], h->sts64[c]) != EP_OK) return EP_ERR_CUDA;
    if (copy_into<T>(h, h->rq[c], h->rq64[c]) != EP_OK) return EP_ERR_CUDA;
  }
  if (h->opts.incompressible) {
    // base pressure step of the incompressible sweep: -K~ div v0 (es64 is
    // free after the start stage); the state starts at p_hat
    const double *v0[3] = {h->H.v0[0], h->H.v0[1], h->H.v0[2]};
    launch_scaled_div(g, v0, -make_scal(h).KDt, h->es64[0], st);
    if (copy_into<T>(h, h->pb, h->es64[0]) != EP_OK) return EP_ERR_CUDA;
  } else if (copy_into<T>(h, h->pb, h->stp64) != EP_OK) {
    return EP_ERR_CUDA;
  }
  if (copy_into<T>(h, h->stp[0], h->stp64) != EP_OK) return EP_ERR_CUDA;
  if (copy_into<T>(h, h->stp[1], h->stp64) != EP_OK) return EP_ERR_CUDA;
  if (copy_into<T>(h, h->cp, h->stp64) != EP_OK) return EP_ERR_CUDA;
  if (copy_into<T>(h, h->yc, h->yc64) != EP_OK) return EP_ERR_CUDA;
  for (int r = 0; r < (nd == 3 ? 2 : 1); ++r)
    if (copy_into<T>(h, h->rd[r], h->rd64[r]) != EP_OK) return EP_ERR_CUDA;
  if (copy_into<T>(h, h->s, h->s64) != EP_OK) return EP_ERR_CUDA;
  CK(h, cudaGetLastError());
  return EP_OK;
}

// The fused 3D kernels serve sweeps without a body force.  AUTO takes the
// register z-march kernel for FP32 grids (the fastest measured on GB300) and
// the staged sweep for FP64 ones (bound by FP64 arithmetic, where the staged
// sweep's lack of halo recomputation wins).
int fused_variant(const ep_grid *h) {
  if (h->variant == EP_KERNEL_AUTO)
    return h->prec == EP_FP32_MIXED ? EP_KERNEL_FUSED_REG : EP_KERNEL_STAGED;
  return h->variant;
}

template <typename T>
bool use_fused(const ep_grid *h) {
  if (h->ndim != 3 || h->have_f || h->Gc) return false;
  const int v = fused_variant(h);
  return v == EP_KERNEL_FUSED || v == EP_KERNEL_FUSED_TMA || v == EP_KERNEL_FUSED_REG;
}

// the check iteration runs fused too: the FP32 register sweep reduces the
// stopping measures itself (the other flavours and FP64 take the staged
// check iteration)
template <typename T>
bool fused_check(const ep_grid *h) {
  return sizeof(T) == 4 && use_fused<T>(h) && fused_variant(h) == EP_KERNEL_FUSED_REG;
}

// one fused 3D iteration in the grid's chosen flavour
template <typename T>
bool launch_fused_any(const ep_grid *h, const Stage<T> &S, DevInfo *di, cudaStream_t st, bool check = false) {
  const int v = fused_variant(h);
  if (v == EP_KERNEL_FUSED_TMA) return launch_fused3d_tma<T>(h->g, S, h->dscal, di, h->kz, st);
  if (v == EP_KERNEL_FUSED_REG) {
    launch_fused3d_reg<T>(h->g, S, h->dscal, di, h->kz, st, check);
    return true;
  }
  launch_fused3d<T>(h->g, S, h->dscal, di, h->kz, st);
  return true;
}

// One chunk of n_chk iterations (first one a check iteration), captured once.
template <typename T>
ep_status capture_chunk(ep_grid *h) {
  if (h->chunk) return EP_OK;
  const Geo &g = h->g;
  cudaGraph_t graph;
  const bool f2 = use_fused2d<T>(h);
  int blocks = 0;
  if (f2) {
    ep_status r = prepare_solo2d<T>(h);
    if (r != EP_OK) return r;
    blocks = std::min(persistent_blocks(h->tile, sizeof(T)),
                      (h->n_items + fused2d_items_per_block(h->tile) - 1) / fused2d_items_per_block(h->tile));
  }
  CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  for (int it = 0; f2 && it < h->opts.n_chk; ++it) {
    launch_fused2d<T>(h->tile, (const Inst2<T> *)h->inst_dev, h->items_dev, h->n_items, it & 1, it == 0, blocks,
                      h->cap);
    if (it == 0) launch_check_batch<T>((const Inst2<T> *)h->inst_dev, 1, h->cap);
  }
  for (int it = 0; !f2 && it < h->opts.n_chk; ++it) {
    Stage<T> S = sweep_stage<T>(h, it & 1);
    const int chk = it == 0;
    if ((!chk || fused_check<T>(h)) && use_fused<T>(h)) {
      if (!launch_fused_any<T>(h, S, h->dinfo, h->cap, chk)) {
        cudaGraph_t gr;
        cudaStreamEndCapture(h->cap, &gr);
        if (gr) cudaGraphDestroy(gr);
        return fail(h, EP_ERR_CUDA, "tensor map encoding failed");
      }
      if (chk) launch_check(h->dinfo, h->dscal, h->cap);
      continue;
    }
    launch_strain<T>(g, S, h->dscal, h->dinfo, h->cap);
    launch_trial<T>(g, S, h->dscal, h->dinfo, h->cap);
    launch_return_centres<T>(g, S, h->dscal, h->dinfo, chk, h->cap);
    launch_return_edges<T>(g, S, h->dscal, h->dinfo, chk, h->cap);
    launch_velocity<T>(g, S, h->dscal, h->dinfo, chk, h->cap);
    if (chk) launch_check(h->dinfo, h->dscal, h->cap);
  }
  cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
  if (e != cudaSuccess) return fail(h, EP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->chunk, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(h, EP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return EP_OK;
}

// Commit the iterate held in sweep buffers (u[0], state[1]).
template <typename T>
ep_status commit(ep_grid *h) {
  const Geo &g = h->g;
  cudaStream_t st = h->stream;
  const T *uf[3] = {P<T>(h->u[0][0]), P<T>(h->u[0][1]), P<T>(h->u[0][2])};
  for (int d = 0; d < h->ndim; ++d)
    CK(h, cudaMemcpyAsync(h->vpp[d], h->H.v[d], g.box * sizeof(double), cudaMemcpyDeviceToDevice, st));
  launch_compose<T>(g, h->H.v0, uf, h->H.v, st);
  Stage<double> S = phys_stage(h, h->H.v);
  launch_strain<double>(g, S, h->dscal, nullptr, st);
  launch_trial<double>(g, S, h->dscal, nullptr, st);
  if (h->wrecord && h->w0) {
    // the physical response of the converged velocity with the old history
    // (warm-start training targets); the trial stays in Tn64 / Ts64
    launch_return_centres<double>(g, S, h->dscal, nullptr, 0, st);
    launch_return_edges<double>(g, S, h->dscal, nullptr, 0, st);
    launch_warm_record(g, h->stn64, h->sts64, h->w0, st);
  }
  CK(h, cudaMemsetAsync(h->dnpl, 0, sizeof(unsigned long long), st));
  const T *stn[3] = {P<T>(h->stn[1][0]), P<T>(h->stn[1][1]), P<T>(h->stn[1][2])};
  const T *sts[3] = {P<T>(h->sts[1][0]), P<T>(h->sts[1][1]), P<T>(h->sts[1][2])};
  launch_commit<T>(g, h->H, h->Tn64, h->Ts64, h->es64, stn, sts, P<T>(h->stp[1]), P<T>(h->s), h->dscal, h->dnpl,
                   st);
  launch_line_integrals(g, h->H, h->dline, st);
  CK(h, cudaGetLastError());
  h->in_increment = false;
  h->solving = false;
  h->n_commits += 1;
  return EP_OK;
}

// Iterate the open increment for at most max_chunks chunks.  The first call
// of an increment starts the convergence record; a call that ends before the
// record is decided returns EP_PENDING and the next call continues the same
// iteration (the state sits in buffer 0 after every whole chunk, n_chk being
// even).  The decided call commits on convergence.
template <typename T>
ep_status solve(ep_grid *h, long long max_chunks, ep_solve_info *info) {
  ep_status r = capture_chunk<T>(h);
  if (r != EP_OK) return r;
  if (!h->solving) {
    DevInfo init{};
    init.max_iter = h->opts.max_iter;
    init.frozen_at = -1;
    *h->hinfo = init;
    CK(h, cudaMemcpyAsync(h->dinfo, h->hinfo, sizeof(DevInfo), cudaMemcpyHostToDevice, h->stream));
    h->solving = true;
  }
  CK(h, cudaEventRecord(h->ev0, h->stream));
  const long long cap = h->opts.max_iter / h->opts.n_chk + 2;
  bool decided = false;
  for (long long c = 0; c < std::min(max_chunks, cap); ++c) {
    CK(h, cudaGraphLaunch(h->chunk, h->stream));
    CK(h, cudaMemcpyAsync(h->hinfo, h->dinfo, sizeof(DevInfo), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->hinfo->done) { decided = true; break; }
  }
  const DevInfo di = *h->hinfo;
  if (!decided) {
    CK(h, cudaEventRecord(h->ev1, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    if (info) {
      memset(info, 0, sizeof(*info));
      info->iters = di.k_check; info->eps_res = di.eps_res; info->eps_mom = di.eps_mom;
      info->eps_tau = di.eps_tau; info->eps_p = di.eps_p; info->eps_rel = di.eps_rel;
      info->max_r = di.max_r; info->max_sigma = di.max_sig; info->ms = ms; info->status = EP_PENDING;
      info->frozen_at = di.frozen_at;
    }
    return EP_PENDING;
  }
  h->solving = false;
  ep_status st = di.done == 1 ? EP_OK : di.done == 2 ? EP_ERR_DIVERGED : di.done == 4 ? EP_ERR_TIMEOUT
                                                                                    : EP_ERR_NOT_CONVERGED;
  unsigned long long npl = 0;
  double line[2] = {0, 0};
  if (st != EP_OK) {
    // keep the last iterate: the next solve continues from stress buffer 0
    const size_t nb = h->g.box * sizeof(T);
    for (int d = 0; d < h->ndim; ++d) CK(h, cudaMemcpyAsync(h->stn[0][d], h->stn[1][d], nb, cudaMemcpyDeviceToDevice, h->stream));
    for (int c = 0; c < n_shear(h->ndim); ++c)
      CK(h, cudaMemcpyAsync(h->sts[0][c], h->sts[1][c], nb, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->stp[0], h->stp[1], nb, cudaMemcpyDeviceToDevice, h->stream));
  }
  if (st == EP_OK) {
    r = commit<T>(h);
    if (r != EP_OK) return r;
    CK(h, cudaMemcpyAsync(&npl, h->dnpl, sizeof(npl), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(line, h->dline, sizeof(line), cudaMemcpyDeviceToHost, h->stream));
  }
  CK(h, cudaEventRecord(h->ev1, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  float ms = 0.f;
  CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  if (info) {
    memset(info, 0, sizeof(*info));
    info->iters = di.iters;
    info->eps_res = di.eps_res; info->eps_mom = di.eps_mom; info->eps_tau = di.eps_tau; info->eps_p = di.eps_p;
    info->eps_rel = di.eps_rel; info->max_r = di.max_r; info->max_sigma = di.max_sig;
    info->n_plastic = (long long)npl;
    info->sxx_int_centre = line[0]; info->sxx_int_right = line[1];
    info->ms = ms;
    info->status = st;
    info->frozen_at = di.frozen_at;
  }
  if (st == EP_ERR_DIVERGED) return fail(h, st, "NaN in a residual norm");
  if (st == EP_ERR_TIMEOUT) return fail(h, st, "a bounded device wait gave up");
  if (st == EP_ERR_NOT_CONVERGED) return fail(h, st, "max_iter reached before eps_res <= tol");
  return EP_OK;
}

}  // namespace

// ============================================================================
extern "C" {

ep_status ep_workspace_bytes(int ndim, const int n[3], ep_precision prec, size_t *bytes) {
  if ((ndim != 2 && ndim != 3) || !n || !bytes || (prec != EP_FP64 && prec != EP_FP32_MIXED))
    return fail(nullptr, EP_ERR_ARG, "ep_workspace_bytes: bad arguments");
  for (int d = 0; d < ndim; ++d)
    if (n[d] < 1) return fail(nullptr, EP_ERR_ARG, "ep_workspace_bytes: n < 1");
  ep_grid tmp;
  tmp.ndim = ndim;
  tmp.prec = prec;
  const double L[3] = {1, 1, 1};
  tmp.g = make_geo(ndim, n, L);
  Arena a;
  carve(&tmp, a);
  *bytes = a.off;
  return EP_OK;
}

ep_status ep_default_solver(int ndim, ep_solver_opts *o) {
  if (!o || (ndim != 2 && ndim != 3)) return fail(nullptr, EP_ERR_ARG, "ep_default_solver: bad arguments");
  o->tol = 1e-8;
  o->max_iter = 10000000;
  o->n_chk = 100;
  o->c_cfl = 0.9 / sqrt((double)ndim);
  o->xi = 1.0;
  o->r_pt = 0.5;
  o->jaumann = 1;
  o->freeze_iter = -1;
  o->freeze_eps = 1e-4;
  o->advection = 0;
  o->incompressible = 0;
  o->wait_cycles = 0;
  return EP_OK;
}

ep_status ep_create_grid(int ndim, const int n[3], const double L[3], ep_precision prec, void *stream,
                         void *workspace, size_t workspace_bytes, ep_handle *out) {
  if (!out || !n || !L || (ndim != 2 && ndim != 3) || (prec != EP_FP64 && prec != EP_FP32_MIXED))
    return fail(nullptr, EP_ERR_ARG, "ep_create_grid: bad arguments");
  *out = nullptr;
  for (int d = 0; d < ndim; ++d)
    if (n[d] < 1 || !(L[d] > 0.0)) return fail(nullptr, EP_ERR_ARG, "ep_create_grid: need n >= 1 and L > 0");
  if (workspace && ((uintptr_t)workspace & 255u))
    return fail(nullptr, EP_ERR_ARG, "ep_create_grid: workspace must be 256-byte aligned");
  ep_grid *h = new ep_grid();
  h->ndim = ndim;
  h->prec = prec;
  for (int d = 0; d < 3; ++d) { h->n[d] = d < ndim ? n[d] : 1; h->L[d] = d < ndim ? L[d] : 1.0; }
  h->g = make_geo(ndim, h->n, h->L);
  ep_default_solver(ndim, &h->opts);
  Arena a;
  carve(h, a);
  h->arena_bytes = a.off;
  cudaError_t e;
  if (workspace) {
    if (workspace_bytes < h->arena_bytes) {
      delete h;
      return fail(nullptr, EP_ERR_OOM, "ep_create_grid: workspace smaller than ep_workspace_bytes");
    }
    h->arena = (char *)workspace;
  } else {
    e = cudaMalloc((void **)&h->arena, h->arena_bytes);
    if (e != cudaSuccess) {
      delete h;
      return fail(nullptr, EP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->own_arena = true;
  }
  a = Arena();
  a.base = h->arena;
  a.dry = false;
  carve(h, a);
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    h->own_stream = true;
    if (e != cudaSuccess) { ep_destroy(h); return fail(nullptr, EP_ERR_CUDA, "cudaStreamCreate failed"); }
  }
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost((void **)&h->hinfo, sizeof(DevInfo)) != cudaSuccess ||
      cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
    ep_destroy(h);
    return fail(nullptr, EP_ERR_CUDA, "ep_create_grid: stream/event/pinned allocation failed");
  }
  if (fused3d_configure() != cudaSuccess || fused2d_configure() != cudaSuccess ||
      fused3d_tma_configure() != cudaSuccess || fused3d_reg_configure() != cudaSuccess) {
    ep_destroy(h);
    return fail(nullptr, EP_ERR_CUDA, "ep_create_grid: fused kernel shared-memory attribute");
  }
  e = cudaMemsetAsync(h->arena, 0, h->arena_bytes, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    ep_destroy(h);
    return fail(nullptr, EP_ERR_CUDA, std::string("ep_create_grid: ") + cudaGetErrorString(e));
  }
  *out = h;
  return EP_OK;
}

ep_status ep_set_material(ep_handle h, double K, double G, double mu_s, double phi_deg, double psi_deg,
                          const double *cohesion) {
  if (!h) return fail(nullptr, EP_ERR_ARG, "null handle");
  if (!(K > 0.0) || !(G > 0.0) || !(mu_s > 0.0) || !cohesion)
    return fail(h, EP_ERR_ARG, "ep_set_material: need K, G, mu_s > 0 and a cohesion array");
  if (psi_deg != 0.0) return fail(h, EP_ERR_ARG, "ep_set_material: the return assumes psi = 0");
  if (!std::isfinite(phi_deg)) return fail(h, EP_ERR_ARG, "ep_set_material: friction angle not finite");
  const long long ncell = (long long)h->g.nx * h->g.ny * h->g.nz;
  for (long long q = 0; q < ncell; ++q)
    if (!std::isfinite(cohesion[q]))
      return fail(h, EP_ERR_ARG, "ep_set_material: cohesion of cell " + std::to_string(q) + " is not finite");
  const double phi = phi_deg * M_PI / 180.0;
  h->K = K; h->G = G; h->mu_s = mu_s;
  if (h->ndim == 2) {
    h->A = sin(phi); h->B = cos(phi);
  } else {
    h->A = 6.0 * sin(phi) / (sqrt(3.0) * (3.0 - sin(phi)));
    h->B = 6.0 * cos(phi) / (sqrt(3.0) * (3.0 - sin(phi)));
  }
  ep_status r = upload_box(h, cohesion, h->H.coh, h->g.nx, h->g.ny, h->g.nz);
  if (r != EP_OK) return r;
  double cm = 0.0;
  for (long long q = 0; q < (long long)h->g.nx * h->g.ny * h->g.nz; ++q) cm = std::max(cm, fabs(cohesion[q]));
  h->cmax = cm > 0.0 ? cm : 1.0;
  h->have_material = true;
  return EP_OK;
}

ep_status ep_set_shear_modulus(ep_handle h, const double *G) {
  if (!h) return fail(nullptr, EP_ERR_ARG, "null handle");
  if (h->in_increment) return fail(h, EP_ERR_STATE, "ep_set_shear_modulus: not allowed inside an open increment");
  const long long ncell = (long long)h->g.nx * h->g.ny * h->g.nz;
  if (h->chunk) { cudaGraphExecDestroy(h->chunk); h->chunk = nullptr; }   // captured stages change
  h->items_tile = -1;
  if (!G) {
    if (h->Gc) {
      cudaFree(h->Gc);
      for (int w = 0; w < 4; ++w) {
        cudaFree(h->ge64[w]); cudaFree(h->gc64[w]);
        if (h->prec != EP_FP64) { cudaFree(h->geT[w]); cudaFree(h->gcT[w]); }
        h->ge64[w] = h->gc64[w] = nullptr; h->geT[w] = h->gcT[w] = nullptr;
      }
    }
    h->Gc = nullptr;
    h->H.te_c = nullptr;
    return EP_OK;
  }
  double gm = 0.0;
  for (long long q = 0; q < ncell; ++q) {
    if (!(G[q] > 0.0) || !std::isfinite(G[q]))
      return fail(h, EP_ERR_ARG, "ep_set_shear_modulus: every value must be finite and > 0");
    gm = std::max(gm, G[q]);
  }
  const size_t nb = h->g.box * sizeof(double), nt = h->g.box * (h->prec == EP_FP64 ? 8 : 4);
  if (!h->Gc) {
    CK(h, cudaMalloc((void **)&h->Gc, nb));
    for (int w = 0; w < 4; ++w) {
      CK(h, cudaMalloc((void **)&h->ge64[w], nb));
      CK(h, cudaMalloc((void **)&h->gc64[w], nb));
      if (h->prec == EP_FP64) { h->geT[w] = h->ge64[w]; h->gcT[w] = h->gc64[w]; }
      else { CK(h, cudaMalloc(&h->geT[w], nt)); CK(h, cudaMalloc(&h->gcT[w], nt)); }
    }
  }
  ep_status r = upload_box(h, G, h->Gc, h->g.nx, h->g.ny, h->g.nz);
  if (r != EP_OK) return r;
  h->Gmax = gm;
  h->H.te_c = h->ge64[0];
  return EP_OK;
}

ep_status ep_set_solver(ep_handle h, const ep_solver_opts *o) {
  if (!h || !o) return fail(h, EP_ERR_ARG, "ep_set_solver: null argument");
  if (!(o->tol >= 0.0) || o->n_chk < 2 || (o->n_chk & 1) || o->max_iter < 0 || o->max_iter % o->n_chk ||
      !(o->c_cfl > 0.0) || !(o->xi > 0.0) || !(o->r_pt > 0.0) || !(o->freeze_eps >= 0.0))
    return fail(h, EP_ERR_ARG, "ep_set_solver: need tol >= 0, even n_chk >= 2, max_iter a multiple of n_chk, "
                               "c_cfl, xi, r_pt > 0, freeze_eps >= 0");
  if (o->n_chk != h->opts.n_chk && h->chunk) {
    cudaGraphExecDestroy(h->chunk);
    h->chunk = nullptr;
  }
  h->opts = *o;
  return EP_OK;
}

// validation, per-increment scalars and the body force of a new increment
static ep_status set_increment(ep_grid *h, const double rates[3], double dt, const double *body_force) {
  if (!h) return fail(nullptr, EP_ERR_ARG, "null handle");
  if (!h->have_material) return fail(h, EP_ERR_STATE, "ep_apply_increment: set the material first");
  if (!(dt > 0.0)) return fail(h, EP_ERR_ARG, "ep_apply_increment: dt must be > 0");
  for (int d = 0; d < 3; ++d) h->rate[d] = d < h->ndim ? rates[d] : 0.0;
  h->dt = dt;
  const Scal sc = make_scal(h);
  CK(h, cudaMemcpyAsync(h->dscal, &sc, sizeof(Scal), cudaMemcpyHostToDevice, h->stream));
  const size_t es = h->prec == EP_FP64 ? 8 : 4;
  if (h->Gc) {
    // per-cell modulus: 2 eta_ve and c2 of every point for this dt
    launch_shear_fields(h->g, h->Gc, h->mu_s, dt, h->ge64, h->gc64, h->stream);
    if (es == 4)
      for (int w = 0; w < 4; ++w) {
        launch_convert<float, double>((float *)h->geT[w], h->ge64[w], h->g.box, h->stream);
        launch_convert<float, double>((float *)h->gcT[w], h->gc64[w], h->g.box, h->stream);
      }
    CK(h, cudaGetLastError());
  }
  CK(h, cudaStreamSynchronize(h->stream));
  if (h->have_f != (body_force != nullptr) && h->chunk) {
    cudaGraphExecDestroy(h->chunk);  // the captured kernels depend on the body force
    h->chunk = nullptr;
  }
  h->have_f = body_force != nullptr;
  size_t off = 0;
  int ex, ey, ez;
  for (int d = 0; d < h->ndim && body_force; ++d) {
    field_extent(h, EP_VX + d, ex, ey, ez);
    ep_status r = upload_box(h, body_force + off, h->Tn64[0], ex, ey, ez);
    if (r != EP_OK) return r;
    if (es == 8) CK(h, cudaMemcpyAsync(h->f[d], h->Tn64[0], h->g.box * 8, cudaMemcpyDeviceToDevice, h->stream));
    else launch_convert<float, double>((float *)h->f[d], h->Tn64[0], h->g.box, h->stream);
    off += (size_t)ex * ey * ez;
  }
  return EP_OK;
}

static ep_status run_prologue(ep_grid *h, const double *const dv[3]) {
  ep_status r = h->prec == EP_FP64 ? prologue<double>(h, dv) : prologue<float>(h, dv);
  if (r != EP_OK) return r;
  CK(h, cudaStreamSynchronize(h->stream));
  h->started = true;
  h->in_increment = true;
  h->solving = false;
  return EP_OK;
}

// start an increment whose start increment dv already lives on the device
static ep_status apply_common_dev(ep_grid *h, const double rates[3], double dt, const double *body_force,
                                  const double *const dv[3]) {
  ep_status r = set_increment(h, rates, dt, body_force);
  if (r != EP_OK) return r;
  return run_prologue(h, dv);
}

// start an increment, with an optional host start increment dv_start
static ep_status apply_common(ep_handle h, const double rates[3], double dt, const double *body_force,
                              const double *dv_start) {
  ep_status r = set_increment(h, rates, dt, body_force);
  if (r != EP_OK) return r;
  const double *dvh[3] = {nullptr, nullptr, nullptr};
  if (dv_start) {
    // Tn64 is free until the prologue's trial stage, which runs after the
    // start-velocity kernel has consumed dv
    size_t off = 0;
    int ex, ey, ez;
    for (int d = 0; d < h->ndim; ++d) {
      field_extent(h, EP_VX + d, ex, ey, ez);
      r = upload_box(h, dv_start + off, h->Tn64[d], ex, ey, ez);
      if (r != EP_OK) return r;
      dvh[d] = h->Tn64[d];
      off += (size_t)ex * ey * ez;
    }
  }
  return run_prologue(h, dvh);
}

static ep_status warm_features_into(ep_grid *h, int f, float *x) {
  int dims[3];
  warm_dims(h, f, dims);
  const WarmScales ws = warm_scales(h);
  if (h->prec == EP_FP64) launch_warm_features<double>(h->g, h->H, h->vpp, P<double>(h->s), ws, f, x, dims, h->stream);
  else launch_warm_features<float>(h->g, h->H, h->vpp, P<float>(h->s), ws, f, x, dims, h->stream);
  CK(h, cudaGetLastError());
  return EP_OK;
}

// start from the network's prediction (device end to end): the velocity
// channels give the start increment at the faces, the stress channels are
// added to the physical response of that start velocity by the prologue
static ep_status apply_warm(ep_grid *h, const double rates[3], double dt, const double *body_force) {
  int dims[3];
  const int f = h->wcoarse;
  warm_dims(h, f, dims);
  // the scales follow this increment's loading
  for (int d = 0; d < 3; ++d) h->rate[d] = d < h->ndim ? rates[d] : 0.0;
  h->dt = dt;
  ep_status r = warm_features_into(h, f, h->wx);
  if (r != EP_OK) return r;
  CK(h, cudaStreamSynchronize(h->stream));
  r = ep_net_forward(h->net, h->wx, 1, dims, h->wy);
  if (r != EP_OK) return fail(h, r, std::string("warm start network: ") + ep_net_last_error(h->net));
  CK(h, cudaDeviceSynchronize());
  const WarmScales ws = warm_scales(h);
  // Tn64 is free until the prologue's trial stage (after the start velocity)
  double *dv[3] = {h->Tn64[0], h->Tn64[1], h->ndim == 3 ? h->Tn64[2] : nullptr};
  launch_warm_dv(h->g, h->wy, f, 1.0 / ws.sv_inv, dv, dims, h->stream);
  CK(h, cudaGetLastError());
  h->warm_stress = true;
  r = apply_common_dev(h, rates, dt, body_force, dv);
  h->warm_stress = false;
  return r;
}

ep_status ep_warm_dims(ep_handle h, int coarsen, int dims[3]) {
  if (!h || !dims || coarsen < 1) return fail(h, EP_ERR_ARG, "ep_warm_dims: bad arguments");
  warm_dims(h, coarsen, dims);
  return EP_OK;
}

ep_status ep_attach_warm_start(ep_handle h, ep_net_handle net, int coarsen) {
  if (!h) return fail(nullptr, EP_ERR_ARG, "null handle");
  if (coarsen < 1) return fail(h, EP_ERR_ARG, "ep_attach_warm_start: coarsen must be >= 1");
  if (h->wx) { cudaFree(h->wx); h->wx = nullptr; }
  if (h->wy) { cudaFree(h->wy); h->wy = nullptr; }
  h->net = net;
  h->wcoarse = coarsen;
  if (!net) return EP_OK;
  int dims[3];
  warm_dims(h, coarsen, dims);
  const long long nv = (long long)dims[0] * dims[1] * dims[2];
  CK(h, cudaMalloc((void **)&h->wx, nv * warm_in_channels(h->ndim) * sizeof(float)));
  CK(h, cudaMalloc((void **)&h->wy, nv * warm_out_channels(h->ndim) * sizeof(float)));
  return EP_OK;
}

ep_status ep_warm_record(ep_handle h, int on) {
  if (!h) return fail(nullptr, EP_ERR_ARG, "null handle");
  if (on && !h->w0) {
    const size_t n = (size_t)(h->ndim + n_shear(h->ndim)) * h->g.box;
    CK(h, cudaMalloc((void **)&h->w0, n * sizeof(float)));
    CK(h, cudaMemset(h->w0, 0, n * sizeof(float)));
  }
  if (!on && h->w0) { cudaFree(h->w0); h->w0 = nullptr; }
  h->wrecord = on != 0;
  return EP_OK;
}

ep_status ep_warm_features(ep_handle h, int coarsen, float *dev_out) {
  if (!h || !dev_out || coarsen < 1) return fail(h, EP_ERR_ARG, "ep_warm_features: bad arguments");
  if (h->n_commits < 2) return fail(h, EP_ERR_STATE, "ep_warm_features: needs two committed increments");
  ep_status r = warm_features_into(h, coarsen, dev_out);
  if (r != EP_OK) return r;
  CK(h, cudaStreamSynchronize(h->stream));
  return EP_OK;
}

ep_status ep_warm_target(ep_handle h, int coarsen, float *dev_out) {
  if (!h || !dev_out || coarsen < 1) return fail(h, EP_ERR_ARG, "ep_warm_target: bad arguments");
  if (!h->wrecord || h->n_commits < 1) return fail(h, EP_ERR_STATE, "ep_warm_target: record a committed increment first");
  int dims[3];
  warm_dims(h, coarsen, dims);
  launch_warm_target(h->g, h->H, h->vpp, h->w0, warm_scales(h), coarsen, dev_out, dims, h->stream);
  CK(h, cudaGetLastError());
  CK(h, cudaStreamSynchronize(h->stream));
  return EP_OK;
}

ep_status ep_apply_increment_rates(ep_handle h, const double rates[3], double dt, const double *body_force,
                                   const double *dv_start) {
  if (!rates) return fail(h, EP_ERR_ARG, "ep_apply_increment_rates: null rates");
  return apply_common(h, rates, dt, body_force, dv_start);
}

ep_status ep_apply_increment(ep_handle h, double a, double dt, int load_plane, const double *body_force,
                             int use_warm_start) {
  if (!h) return fail(nullptr, EP_ERR_ARG, "null handle");
  double r[3] = {0, 0, 0};
  if (load_plane == EP_LOAD_XY) { r[0] = a; r[1] = -a; }
  else if (load_plane == EP_LOAD_XZ && h->ndim == 3) { r[0] = a; r[2] = -a; }
  else return fail(h, EP_ERR_ARG, "ep_apply_increment: load_plane must be EP_LOAD_XY, or EP_LOAD_XZ in 3D");
  if (use_warm_start && !h->net) return fail(h, EP_ERR_STATE, "ep_apply_increment: no warm-start network attached");
  if (use_warm_start && h->n_commits >= 2) return apply_warm(h, r, dt, body_force);
  return apply_common(h, r, dt, body_force, nullptr);
}

ep_status ep_solve_increment(ep_handle h, ep_solve_info *info) {
  if (!h) return fail(nullptr, EP_ERR_ARG, "null handle");
  if (!h->in_increment) return fail(h, EP_ERR_STATE, "ep_solve_increment: apply an increment first");
  const long long all = 1ll << 62;
  return h->prec == EP_FP64 ? solve<double>(h, all, info) : solve<float>(h, all, info);
}

ep_status ep_solve_chunks(ep_handle h, int max_chunks, ep_solve_info *info) {
  if (!h || max_chunks < 1) return fail(h, EP_ERR_ARG, "ep_solve_chunks: null handle or max_chunks < 1");
  if (!h->in_increment) return fail(h, EP_ERR_STATE, "ep_solve_chunks: apply an increment first");
  return h->prec == EP_FP64 ? solve<double>(h, max_chunks, info) : solve<float>(h, max_chunks, info);
}

ep_status ep_commit_increment(ep_handle h) {
  if (!h) return fail(nullptr, EP_ERR_ARG, "null handle");
  if (!h->in_increment) return fail(h, EP_ERR_STATE, "ep_commit_increment: no open increment");
  ep_status r = h->prec == EP_FP64 ? commit<double>(h) : commit<float>(h);
  if (r != EP_OK) return r;
  CK(h, cudaStreamSynchronize(h->stream));
  return EP_OK;
}

ep_status ep_field_count(ep_handle h, int f, size_t *count) {
  if (!h || !count) return fail(h, EP_ERR_ARG, "ep_field_count: null argument");
  int ex, ey, ez;
  if (!field_extent(h, f, ex, ey, ez)) return fail(h, EP_ERR_ARG, "ep_field_count: unknown field for this grid");
  *count = (size_t)ex * ey * ez;
  return EP_OK;
}

ep_status ep_get_fields(ep_handle h, int f, double *out, size_t count) {
  if (!h || !out) return fail(h, EP_ERR_ARG, "ep_get_fields: null argument");
  int ex, ey, ez;
  if (!field_extent(h, f, ex, ey, ez) || count != (size_t)ex * ey * ez)
    return fail(h, EP_ERR_ARG, "ep_get_fields: unknown field or wrong count");
  if (f == EP_EII) {
    // sqrt(eps:eps/2) of the accumulated strain, shear averaged to centres
    const int nd = h->ndim;
    std::vector<std::vector<double>> c(6);
    int fx[6] = {EP_EXX, EP_EYY, EP_EZZ, EP_EXY, EP_EXZ, EP_EYZ};
    for (int q = 0; q < 6; ++q) {
      size_t nq;
      if (ep_field_count(h, fx[q], &nq) != EP_OK) continue;
      c[q].resize(nq);
      ep_status r = ep_get_fields(h, fx[q], c[q].data(), nq);
      if (r != EP_OK) return r;
    }
    const int nx = h->g.nx, ny = h->g.ny, nz = h->g.nz;
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          size_t cc = ((size_t)k * ny + j) * nx + i;
          double sq = 0.0;
          for (int d = 0; d < nd; ++d) sq += 0.5 * c[d][cc] * c[d][cc];
          auto xy = [&](int ii, int jj, int kk) { return c[3][((size_t)kk * (ny + 1) + jj) * (nx + 1) + ii]; };
          double exy = 0.25 * (xy(i, j, k) + xy(i + 1, j, k) + xy(i, j + 1, k) + xy(i + 1, j + 1, k));
          sq += exy * exy;
          if (nd == 3) {
            auto xz = [&](int ii, int jj, int kk) { return c[4][((size_t)kk * ny + jj) * (nx + 1) + ii]; };
            auto yz = [&](int ii, int jj, int kk) { return c[5][((size_t)kk * (ny + 1) + jj) * nx + ii]; };
            double exz = 0.25 * (xz(i, j, k) + xz(i + 1, j, k) + xz(i, j, k + 1) + xz(i + 1, j, k + 1));
            double eyz = 0.25 * (yz(i, j, k) + yz(i, j + 1, k) + yz(i, j, k + 1) + yz(i, j + 1, k + 1));
            sq += exz * exz + eyz * eyz;
          }
          out[cc] = sqrt(sq);
        }
    return EP_OK;
  }
  if (f == EP_SCALE) {
    if (h->prec == EP_FP64) {
      CK(h, cudaMemcpyAsync(h->Tn64[0], h->s, h->g.box * 8, cudaMemcpyDeviceToDevice, h->stream));
    } else {
      launch_convert<double, float>(h->Tn64[0], (const float *)h->s, h->g.box, h->stream);
    }
    return download_box(h, h->Tn64[0], out, ex, ey, ez);
  }
  double *box = history_ptr(h, f);
  if (!box) return fail(h, EP_ERR_ARG, "ep_get_fields: field not stored");
  return download_box(h, box, out, ex, ey, ez);
}

ep_status ep_set_fields(ep_handle h, int f, const double *in, size_t count) {
  if (!h || !in) return fail(h, EP_ERR_ARG, "ep_set_fields: null argument");
  int ex, ey, ez;
  if (!field_extent(h, f, ex, ey, ez) || count != (size_t)ex * ey * ez || f == EP_EII || f == EP_SCALE ||
      f == EP_V0X || f == EP_V0Y || f == EP_V0Z)
    return fail(h, EP_ERR_ARG, "ep_set_fields: not a settable history field, or wrong count");
  if (h->in_increment) return fail(h, EP_ERR_STATE, "ep_set_fields: not allowed inside an open increment");
  ep_status r = upload_box(h, in, history_ptr(h, f), ex, ey, ez);
  if (r != EP_OK) return r;
  if (f == EP_VX || f == EP_VY || f == EP_VZ) h->started = true;
  return EP_OK;
}

static std::vector<double *> history_arrays(ep_grid *h) {
  std::vector<double *> v;
  const int nd = h->ndim, ns = n_shear(nd);
  for (int d = 0; d < nd; ++d) {
    v.push_back(h->H.v[d]); v.push_back(h->H.tn[d]); v.push_back(h->H.u[d]); v.push_back(h->H.an[d]);
    v.push_back(h->vpp[d]);  // the warm start's previous increment
  }
  for (int c = 0; c < ns; ++c) { v.push_back(h->H.ts[c]); v.push_back(h->H.as[c]); }
  v.push_back(h->H.p);
  v.push_back(h->H.epl);
  return v;
}

ep_status ep_snapshot(ep_handle h) {
  if (!h) return fail(nullptr, EP_ERR_ARG, "null handle");
  auto arr = history_arrays(h);
  const size_t nb = h->g.box * sizeof(double);
  // plus the last return scale (sweep type), a feature of the warm start
  const size_t ns = h->g.box * (h->prec == EP_FP64 ? sizeof(double) : sizeof(float));
  if (!h->snap) CK(h, cudaMalloc((void **)&h->snap, nb * arr.size() + ns));
  for (size_t q = 0; q < arr.size(); ++q)
    CK(h, cudaMemcpyAsync(h->snap + q * nb, arr[q], nb, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaMemcpyAsync(h->snap + arr.size() * nb, h->s, ns, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  h->snap_started = h->started;
  h->snap_commits = h->n_commits;
  h->snap_adv_done = h->adv_done;
  return EP_OK;
}

ep_status ep_restore(ep_handle h) {
  if (!h) return fail(nullptr, EP_ERR_ARG, "null handle");
  if (!h->snap) return fail(h, EP_ERR_STATE, "ep_restore: no snapshot taken");
  auto arr = history_arrays(h);
  const size_t nb = h->g.box * sizeof(double);
  const size_t ns = h->g.box * (h->prec == EP_FP64 ? sizeof(double) : sizeof(float));
  for (size_t q = 0; q < arr.size(); ++q)
    CK(h, cudaMemcpyAsync(arr[q], h->snap + q * nb, nb, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaMemcpyAsync(h->s, h->snap + arr.size() * nb, ns, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  h->started = h->snap_started;
  h->n_commits = h->snap_commits;
  h->adv_done = h->snap_adv_done;   // a restored history is advected again
  h->in_increment = false;
  h->solving = false;
  return EP_OK;
}

ep_status ep_time_sweep(ep_handle h, int iters, double *ms_out, int n_out, int *n_kernels) {
  if (!h || iters < 1 || !ms_out || n_out < 1) return fail(h, EP_ERR_ARG, "ep_time_sweep: bad arguments");
  if (!h->have_material || h->dt <= 0.0) return fail(h, EP_ERR_STATE, "ep_time_sweep: apply an increment first");
  const int nk = 5;
  std::vector<cudaEvent_t> ev(nk + 1);
  for (auto &e : ev) CK(h, cudaEventCreate(&e));
  std::vector<double> acc(nk + 1, 0.0);
  const bool f2 = h->prec == EP_FP64 ? use_fused2d<double>(h) : use_fused2d<float>(h);
  if (f2) {
    ep_status r = h->prec == EP_FP64 ? prepare_solo2d<double>(h) : prepare_solo2d<float>(h);
    if (r != EP_OK) return r;
    const size_t el = h->prec == EP_FP64 ? 8 : 4;
    const int blocks = std::min(persistent_blocks(h->tile, el), (h->n_items + fused2d_items_per_block(h->tile) - 1) /
                                                                    fused2d_items_per_block(h->tile));
    // clear the record of the last solve (a converged grid would be skipped)
    if (el == 8) launch_init_batch<double>((const Inst2<double> *)h->inst_dev, 1, 0, h->stream);
    else launch_init_batch<float>((const Inst2<float> *)h->inst_dev, 1, 0, h->stream);
    for (int it = 0; it < iters; ++it) {
      CK(h, cudaEventRecord(ev[0], h->stream));
      if (el == 8)
        launch_fused2d<double>(h->tile, (const Inst2<double> *)h->inst_dev, h->items_dev, h->n_items, it & 1, 0,
                               blocks, h->stream);
      else
        launch_fused2d<float>(h->tile, (const Inst2<float> *)h->inst_dev, h->items_dev, h->n_items, it & 1, 0,
                              blocks, h->stream);
      CK(h, cudaEventRecord(ev[1], h->stream));
      CK(h, cudaGetLastError());
      CK(h, cudaEventSynchronize(ev[1]));
      float ms = 0.f;
      CK(h, cudaEventElapsedTime(&ms, ev[0], ev[1]));
      acc[0] += ms;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    ms_out[0] = acc[0] / iters;
    if (n_out > 1) ms_out[1] = acc[0] / iters;
    if (n_kernels) *n_kernels = 1;
    h->in_increment = false;
    h->solving = false;
    return EP_OK;
  }
  const bool fused = h->prec == EP_FP64 ? use_fused<double>(h) : use_fused<float>(h);
  if (fused) {
    for (int it = 0; it < iters; ++it) {
      CK(h, cudaEventRecord(ev[0], h->stream));
      bool ok = h->prec == EP_FP64 ? launch_fused_any<double>(h, sweep_stage<double>(h, it & 1), nullptr, h->stream)
                                   : launch_fused_any<float>(h, sweep_stage<float>(h, it & 1), nullptr, h->stream);
      if (!ok) return fail(h, EP_ERR_CUDA, "tensor map encoding failed");
      CK(h, cudaEventRecord(ev[1], h->stream));
      CK(h, cudaGetLastError());
      CK(h, cudaEventSynchronize(ev[1]));
      float ms = 0.f;
      CK(h, cudaEventElapsedTime(&ms, ev[0], ev[1]));
      acc[0] += ms;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    ms_out[0] = acc[0] / iters;
    if (n_out > 1) ms_out[1] = acc[0] / iters;
    if (n_kernels) *n_kernels = 1;
    h->in_increment = false;
    h->solving = false;
    return EP_OK;
  }
  for (int it = 0; it < iters; ++it) {
    const int b = it & 1;
    CK(h, cudaEventRecord(ev[0], h->stream));
    if (h->prec == EP_FP64) {
      Stage<double> S = sweep_stage<double>(h, b);
      launch_strain<double>(h->g, S, h->dscal, nullptr, h->stream); CK(h, cudaEventRecord(ev[1], h->stream));
      launch_trial<double>(h->g, S, h->dscal, nullptr, h->stream); CK(h, cudaEventRecord(ev[2], h->stream));
      launch_return_centres<double>(h->g, S, h->dscal, nullptr, 0, h->stream); CK(h, cudaEventRecord(ev[3], h->stream));
      launch_return_edges<double>(h->g, S, h->dscal, nullptr, 0, h->stream); CK(h, cudaEventRecord(ev[4], h->stream));
      launch_velocity<double>(h->g, S, h->dscal, nullptr, 0, h->stream); CK(h, cudaEventRecord(ev[5], h->stream));
    } else {
      Stage<float> S = sweep_stage<float>(h, b);
      launch_strain<float>(h->g, S, h->dscal, nullptr, h->stream); CK(h, cudaEventRecord(ev[1], h->stream));
      launch_trial<float>(h->g, S, h->dscal, nullptr, h->stream); CK(h, cudaEventRecord(ev[2], h->stream));
      launch_return_centres<float>(h->g, S, h->dscal, nullptr, 0, h->stream); CK(h, cudaEventRecord(ev[3], h->stream));
      launch_return_edges<float>(h->g, S, h->dscal, nullptr, 0, h->stream); CK(h, cudaEventRecord(ev[4], h->stream));
      launch_velocity<float>(h->g, S, h->dscal, nullptr, 0, h->stream); CK(h, cudaEventRecord(ev[5], h->stream));
    }
    CK(h, cudaGetLastError());
    CK(h, cudaEventSynchronize(ev[nk]));
    for (int q = 0; q < nk; ++q) {
      float ms = 0.f;
      CK(h, cudaEventElapsedTime(&ms, ev[q], ev[q + 1]));
      acc[q] += ms;
    }
    float tot = 0.f;
    CK(h, cudaEventElapsedTime(&tot, ev[0], ev[nk]));
    acc[nk] += tot;
  }
  for (auto &e : ev) cudaEventDestroy(e);
  for (int q = 0; q < n_out && q <= nk; ++q) ms_out[q] = acc[q] / iters;
  if (n_kernels) *n_kernels = nk;
  h->in_increment = false;  // the sweep state was overwritten
  h->solving = false;
  return EP_OK;
}

ep_status ep_set_kernel(ep_handle h, int variant, int shape) {
  if (!h) return fail(nullptr, EP_ERR_ARG, "null handle");
  if (variant < EP_KERNEL_AUTO || variant > EP_KERNEL_FUSED_REG)
    return fail(h, EP_ERR_ARG, "ep_set_kernel: unknown variant");
  if ((variant == EP_KERNEL_FUSED_TMA || variant == EP_KERNEL_FUSED_REG) && h->ndim != 3)
    return fail(h, EP_ERR_ARG, "ep_set_kernel: the TMA and register sweeps are 3D only");
  if (shape >= 0 && h->ndim == 2 && shape >= FUSED2D_TILES)
    return fail(h, EP_ERR_ARG, "ep_set_kernel: shape is z-planes (3D, 0: by grid size) or a tile 0..2 (2D)");
  if (h->chunk) {
    cudaGraphExecDestroy(h->chunk);
    h->chunk = nullptr;
  }
  h->variant = variant;
  if (shape >= 0) {
    if (h->ndim == 3) h->kz = shape; else h->tile = shape;
  }
  return EP_OK;
}

ep_status ep_sweep_bytes_per_cell(ep_handle h, double *bytes) {
  if (!h || !bytes) return fail(h, EP_ERR_ARG, "ep_sweep_bytes_per_cell: null argument");
  // reads: velocity increment (nd), stress state (nd + ns), pressure, base
  // trial (nd + ns), base pressure, B c, rotation weights (ns + nd - 1);
  // writes: velocity increment, stress state, pressure
  const int nd = h->ndim, ns = n_shear(nd);
  const double words = (nd + (nd + ns) + 1 + (nd + ns) + 1 + 1 + (ns + nd - 1)) + (nd + (nd + ns) + 1);
  *bytes = words * (h->prec == EP_FP64 ? 8.0 : 4.0);
  return EP_OK;
}

}  // extern "C"

struct ep_batch {
  std::vector<ep_grid *> g;
  int count = 0;
  ep_precision prec = EP_FP64;
  cudaStream_t stream = nullptr, cap = nullptr;
  int tile = 0, blocks = 1, n_items = 0;
  void *insts = nullptr;
  int4 *items = nullptr;
  DevInfo *dinfo = nullptr, *hinfo = nullptr;
  cudaGraphExec_t chunk = nullptr;
  int chunk_nchk = 0;          // n_chk the captured chunk was built with
  double dt = 0.0;
  std::vector<double> a;
  std::string err;
};

static ep_status bfail(ep_batch *b, ep_status st, const std::string &m) {
  if (b) b->err = m;
  g_thread_err = m;
  return st;
}

#define BCK(b, call)                                                                                \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return bfail((b), EP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace {

template <typename T>
ep_status batch_upload(ep_batch *b) {
  std::vector<Inst2<T>> I(b->count);
  std::vector<int4> items;
  for (int q = 0; q < b->count; ++q) {
    I[q] = make_inst<T>(b->g[q], b->dinfo + q);
    append_items(items, q, b->g[q]->g, b->tile);
  }
  if (b->items) cudaFree(b->items);
  b->items = nullptr;
  BCK(b, cudaMalloc((void **)&b->items, items.size() * sizeof(int4)));
  BCK(b, cudaMemcpy(b->insts, I.data(), I.size() * sizeof(Inst2<T>), cudaMemcpyHostToDevice));
  BCK(b, cudaMemcpy(b->items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
  b->n_items = (int)items.size();
  b->blocks = std::min(persistent_blocks(b->tile, sizeof(T)),
                       (b->n_items + fused2d_items_per_block(b->tile) - 1) / fused2d_items_per_block(b->tile));
  if (b->chunk) { cudaGraphExecDestroy(b->chunk); b->chunk = nullptr; }
  return EP_OK;
}

// A pair of CUDA events destroyed on every exit path.
struct EventPair {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t create() {
    cudaError_t e = cudaEventCreate(&e0);
    return e == cudaSuccess ? cudaEventCreate(&e1) : e;
  }
  ~EventPair() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// The chunk graph holds n_chk sweeps; every member must use the same n_chk
// (ep_set_solver may have changed one since ep_create_batch), and a chunk
// captured with another n_chk is rebuilt.  The iteration cap (max_iter) is
// taken from the first grid.
template <typename T>
ep_status batch_capture(ep_batch *b) {
  const int nchk = b->g[0]->opts.n_chk;
  for (int q = 1; q < b->count; ++q)
    if (b->g[q]->opts.n_chk != nchk)
      return bfail(b, EP_ERR_STATE, "batch solve: the grids' n_chk differ (ep_set_solver changed one after ep_create_batch)");
  if (b->chunk && b->chunk_nchk == nchk) return EP_OK;
  if (b->chunk) { cudaGraphExecDestroy(b->chunk); b->chunk = nullptr; }
  cudaGraph_t graph;
  BCK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  for (int it = 0; it < nchk; ++it) {
    launch_fused2d<T>(b->tile, (const Inst2<T> *)b->insts, b->items, b->n_items, it & 1, it == 0, b->blocks, b->cap);
    if (it == 0) launch_check_batch<T>((const Inst2<T> *)b->insts, b->count, b->cap);
  }
  cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
  if (e != cudaSuccess) return bfail(b, EP_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->chunk, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(b, EP_ERR_CUDA, std::string("batch instantiate: ") + cudaGetErrorString(e));
  b->chunk_nchk = nchk;
  return EP_OK;
}

template <typename T>
ep_status batch_solve(ep_batch *b, ep_solve_info *infos) {
  ep_status r = batch_capture<T>(b);
  if (r != EP_OK) return r;
  EventPair ev;
  BCK(b, ev.create());
  cudaEvent_t e0 = ev.e0, e1 = ev.e1;
  launch_init_batch<T>((const Inst2<T> *)b->insts, b->count, b->g[0]->opts.max_iter, b->stream);
  BCK(b, cudaEventRecord(e0, b->stream));
  const long long max_chunks = b->g[0]->opts.max_iter / b->g[0]->opts.n_chk + 2;
  for (long long c = 0; c < max_chunks; ++c) {
    BCK(b, cudaGraphLaunch(b->chunk, b->stream));
    BCK(b, cudaMemcpyAsync(b->hinfo, b->dinfo, b->count * sizeof(DevInfo), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    bool all = true;
    for (int q = 0; q < b->count; ++q) all = all && b->hinfo[q].done != 0;
    if (all) break;
  }
  BCK(b, cudaEventRecord(e1, b->stream));
  BCK(b, cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  ep_status worst = EP_OK;
  for (int q = 0; q < b->count; ++q) {
    ep_grid *h = b->g[q];
    const DevInfo di = b->hinfo[q];
    ep_status st = di.done == 1 ? EP_OK : di.done == 2 ? EP_ERR_DIVERGED : EP_ERR_NOT_CONVERGED;
    unsigned long long npl = 0;
    double line[2] = {0, 0};
    if (st == EP_OK) {
      r = commit<T>(h);
      if (r != EP_OK) return bfail(b, r, h->err);
      BCK(b, cudaMemcpyAsync(&npl, h->dnpl, sizeof(npl), cudaMemcpyDeviceToHost, h->stream));
      BCK(b, cudaMemcpyAsync(line, h->dline, sizeof(line), cudaMemcpyDeviceToHost, h->stream));
      BCK(b, cudaStreamSynchronize(h->stream));
    } else if (worst == EP_OK || st == EP_ERR_DIVERGED) {
      worst = st;
    }
    if (infos) {
      ep_solve_info &f = infos[q];
      memset(&f, 0, sizeof(f));
      f.iters = di.iters; f.eps_res = di.eps_res; f.eps_mom = di.eps_mom; f.eps_tau = di.eps_tau;
      f.eps_p = di.eps_p; f.eps_rel = di.eps_rel; f.max_r = di.max_r; f.max_sigma = di.max_sig;
      f.n_plastic = (long long)npl; f.sxx_int_centre = line[0]; f.sxx_int_right = line[1];
      f.ms = ms; f.status = st; f.frozen_at = di.frozen_at;
    }
  }
  if (worst != EP_OK) return bfail(b, worst, "some grids of the batch did not converge");
  return EP_OK;
}

template <typename T>
ep_status batch_restart(ep_batch *b) {
  for (int q = 0; q < b->count; ++q) {
    ep_grid *h = b->g[q];
    h->in_increment = false;
    h->solving = false;
    ep_status r = apply_common(h, h->rate, b->dt, nullptr, nullptr);
    if (r != EP_OK) return bfail(b, r, h->err);
  }
  return EP_OK;
}

}  // namespace

extern "C" {

ep_status ep_create_batch(const ep_handle *grids, int count, ep_batch_handle *out) {
  if (!grids || count < 1 || !out) return bfail(nullptr, EP_ERR_ARG, "ep_create_batch: bad arguments");
  *out = nullptr;
  for (int q = 0; q < count; ++q) {
    if (!grids[q] || grids[q]->ndim != 2) return bfail(nullptr, EP_ERR_ARG, "ep_create_batch: grids must be 2D");
    if (grids[q]->prec != grids[0]->prec || grids[q]->opts.n_chk != grids[0]->opts.n_chk)
      return bfail(nullptr, EP_ERR_ARG, "ep_create_batch: grids must share precision and n_chk");
  }
  ep_batch *b = new ep_batch();
  b->count = count;
  b->prec = grids[0]->prec;
  b->stream = grids[0]->stream;
  for (int q = 0; q < count; ++q) b->g.push_back(grids[q]);
  const size_t isz = b->prec == EP_FP64 ? sizeof(Inst2<double>) : sizeof(Inst2<float>);
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&b->insts, isz * count) != cudaSuccess ||
      cudaMalloc((void **)&b->dinfo, sizeof(DevInfo) * count) != cudaSuccess ||
      cudaMallocHost((void **)&b->hinfo, sizeof(DevInfo) * count) != cudaSuccess) {
    ep_destroy_batch(b);
    return bfail(nullptr, EP_ERR_OOM, "ep_create_batch: allocation failed");
  }
  ep_status r = b->prec == EP_FP64 ? batch_upload<double>(b) : batch_upload<float>(b);
  if (r != EP_OK) { ep_destroy_batch(b); return r; }
  *out = b;
  return EP_OK;
}

ep_status ep_batch_apply_increment(ep_batch_handle b, const double *a, double dt) {
  if (!b || !a) return bfail(b, EP_ERR_ARG, "ep_batch_apply_increment: null argument");
  b->dt = dt;
  for (int q = 0; q < b->count; ++q) {
    const double r[3] = {a[q], -a[q], 0.0};
    ep_status st = apply_common(b->g[q], r, dt, nullptr, nullptr);
    if (st != EP_OK) return bfail(b, st, b->g[q]->err);
  }
  return EP_OK;
}

ep_status ep_batch_solve_increment(ep_batch_handle b, ep_solve_info *infos) {
  if (!b) return bfail(nullptr, EP_ERR_ARG, "null batch");
  for (int q = 0; q < b->count; ++q)
    if (!b->g[q]->in_increment) return bfail(b, EP_ERR_STATE, "ep_batch_solve_increment: apply an increment first");
  return b->prec == EP_FP64 ? batch_solve<double>(b, infos) : batch_solve<float>(b, infos);
}

ep_status ep_batch_set_tile(ep_batch_handle b, int tile) {
  if (!b || tile < 0 || tile >= FUSED2D_TILES) return bfail(b, EP_ERR_ARG, "ep_batch_set_tile: tile must be 0..4");
  b->tile = tile;
  return b->prec == EP_FP64 ? batch_upload<double>(b) : batch_upload<float>(b);
}

ep_status ep_batch_autotune(ep_batch_handle b, int iters, int *tile_out) {
  if (!b || iters < 1) return bfail(b, EP_ERR_ARG, "ep_batch_autotune: bad arguments");
  for (int q = 0; q < b->count; ++q)
    if (!b->g[q]->in_increment) return bfail(b, EP_ERR_STATE, "ep_batch_autotune: apply an increment first");
  EventPair ev;
  BCK(b, ev.create());
  cudaEvent_t e0 = ev.e0, e1 = ev.e1;
  float best = 1e30f;
  int best_tile = 0;
  for (int tile = 0; tile < FUSED2D_TILES; ++tile) {
    b->tile = tile;
    ep_status r = b->prec == EP_FP64 ? batch_upload<double>(b) : batch_upload<float>(b);
    if (r != EP_OK) return r;
    // clear the records of the last solve (a converged grid would be skipped)
    if (b->prec == EP_FP64) launch_init_batch<double>((const Inst2<double> *)b->insts, b->count, 0, b->stream);
    else launch_init_batch<float>((const Inst2<float> *)b->insts, b->count, 0, b->stream);
    // one untimed sweep, then `iters` timed sweeps without checks
    for (int it = 0; it <= iters; ++it) {
      if (it == 1) BCK(b, cudaEventRecord(e0, b->stream));
      if (b->prec == EP_FP64)
        launch_fused2d<double>(tile, (const Inst2<double> *)b->insts, b->items, b->n_items, it & 1, 0, b->blocks, b->stream);
      else
        launch_fused2d<float>(tile, (const Inst2<float> *)b->insts, b->items, b->n_items, it & 1, 0, b->blocks, b->stream);
    }
    BCK(b, cudaEventRecord(e1, b->stream));
    BCK(b, cudaEventSynchronize(e1));
    BCK(b, cudaGetLastError());
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; best_tile = tile; }
  }
  b->tile = best_tile;
  ep_status r = b->prec == EP_FP64 ? batch_upload<double>(b) : batch_upload<float>(b);
  if (r != EP_OK) return r;
  if (tile_out) *tile_out = best_tile;
  // the timed sweeps advanced the iterates: start the increments again
  return b->prec == EP_FP64 ? batch_restart<double>(b) : batch_restart<float>(b);
}

ep_status ep_batch_time_sweep(ep_batch_handle b, int iters, double *ms_per_sweep) {
  if (!b || iters < 1 || !ms_per_sweep) return bfail(b, EP_ERR_ARG, "ep_batch_time_sweep: bad arguments");
  for (int q = 0; q < b->count; ++q)
    if (!b->g[q]->in_increment) return bfail(b, EP_ERR_STATE, "ep_batch_time_sweep: apply an increment first");
  ep_status r = b->prec == EP_FP64 ? batch_upload<double>(b) : batch_upload<float>(b);
  if (r != EP_OK) return r;
  // clear the records of the last solve (a converged grid would be skipped)
  if (b->prec == EP_FP64) launch_init_batch<double>((const Inst2<double> *)b->insts, b->count, 0, b->stream);
  else launch_init_batch<float>((const Inst2<float> *)b->insts, b->count, 0, b->stream);
  EventPair ev;
  BCK(b, ev.create());
  cudaEvent_t e0 = ev.e0, e1 = ev.e1;
  for (int it = 0; it <= iters; ++it) {   // one untimed sweep, then `iters` timed ones
    if (it == 1) BCK(b, cudaEventRecord(e0, b->stream));
    if (b->prec == EP_FP64)
      launch_fused2d<double>(b->tile, (const Inst2<double> *)b->insts, b->items, b->n_items, it & 1, 0, b->blocks,
                             b->stream);
    else
      launch_fused2d<float>(b->tile, (const Inst2<float> *)b->insts, b->items, b->n_items, it & 1, 0, b->blocks,
                            b->stream);
  }
  BCK(b, cudaEventRecord(e1, b->stream));
  BCK(b, cudaEventSynchronize(e1));
  BCK(b, cudaGetLastError());
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  *ms_per_sweep = (double)ms / iters;
  // the timed sweeps advanced the iterates: start the increments again
  return b->prec == EP_FP64 ? batch_restart<double>(b) : batch_restart<float>(b);
}

ep_status ep_destroy_batch(ep_batch_handle b) {
  if (!b) return EP_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->chunk) cudaGraphExecDestroy(b->chunk);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->insts) cudaFree(b->insts);
  if (b->items) cudaFree(b->items);
  if (b->dinfo) cudaFree(b->dinfo);
  if (b->hinfo) cudaFreeHost(b->hinfo);
  delete b;
  return EP_OK;
}

ep_status ep_destroy(ep_handle h) {
  if (!h) return EP_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->chunk) cudaGraphExecDestroy(h->chunk);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->hinfo) cudaFreeHost(h->hinfo);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  if (h->own_arena && h->arena) cudaFree(h->arena);
  if (h->snap) cudaFree(h->snap);
  if (h->wx) cudaFree(h->wx);   // warm-start network input / output
  if (h->wy) cudaFree(h->wy);
  if (h->w0) cudaFree(h->w0);
  if (h->Gc) {
    cudaFree(h->Gc);
    for (int w = 0; w < 4; ++w) {
      cudaFree(h->ge64[w]); cudaFree(h->gc64[w]);
      if (h->prec != EP_FP64) { cudaFree(h->geT[w]); cudaFree(h->gcT[w]); }
    }
  }
  delete h;
  return EP_OK;
}

const char *ep_last_error(ep_handle h) { return h ? h->err.c_str() : g_thread_err.c_str(); }

}  // extern "C"
