// ep_unet.cu -- the learned warm start: a small convolutional U-Net that
// predicts an increment's velocity change from the previous increments, with
// hand-written forward, backward and optimiser kernels.
//
// Network (D = 2 or 3 spatial dimensions, activations NC[Z]YX in FP32,
// weights BF16 with FP32 master copies):
//   level l = 0..L-1 : conv3(c_{l-1} -> c_l) + ReLU, conv3(c_l -> c_l) + ReLU
//                      (c_l = base * 2^l), average-pool by 2 between levels;
//   decoder          : nearest upsample, concatenate the skip of the same
//                      level, two conv3 + ReLU;
//   head             : conv1 (c_0 -> out), no activation, zero-initialised.
// The prediction is added to a baseline chosen by the caller (the previous
// increment's velocity change), so an untrained network reproduces it.
// Training: MSE loss, Adam.  The convolutions run on CUDA cores with FP32
// accumulation: at the sizes used (<= 128 channels) they are a small part of
// an increment's solve time.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "ep_internal.cuh"

namespace ep {

// ep_conv_tc.cu
bool conv_tc_supported(int k, int cout);
int conv_tc_cinp(int cin);
void conv_tc_to_channels_last(const float *x, int N, int C, long long nv, int cp, __nv_bfloat16 *out,
                              cudaStream_t st);
void conv_tc_pack_weights(const __nv_bfloat16 *w, int cin, int cout, int taps, __nv_bfloat16 *out, cudaStream_t st);
cudaError_t conv_tc_forward(int D, const __nv_bfloat16 *xcl, int N, int X, int Y, int Z, int cin,
                            const __nv_bfloat16 *wpk, const float *bias, int cout, int relu, float *y, int *err,
                            cudaStream_t st);

namespace {

constexpr int NT = 256;

inline unsigned nblk(long long n) { return (unsigned)((n + NT - 1) / NT); }

// ---- direct convolution (3^D or 1^D taps), zero padding -------------------
// y[n, co, p] = b[co] + sum_{ci, tap} W(co, ci, tap) x[n, ci, p + tap - r]
// TRANS = true computes the data gradient: channels swapped and taps
// mirrored, i.e. dx = conv(dy, W^T flipped); then b is unused.
template <int D, int K, bool TRANS>
__global__ void k_conv(const float *__restrict__ x, const __nv_bfloat16 *__restrict__ w, const float *__restrict__ b,
                       float *__restrict__ y, int N, int cin, int cout, int X, int Y, int Z, int relu,
                       int w_cin, int w_cout) {
  // one thread per output voxel, a chunk of 8 output channels per blockIdx.y
  constexpr int CB = 8;
  constexpr int R = K / 2;
  const long long nvox = (long long)X * Y * Z;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int co0 = blockIdx.y * CB;
  const int n = blockIdx.z;
  if (t >= nvox) return;
  const int ix = (int)(t % X), iy = (int)((t / X) % Y), iz = (int)(t / ((long long)X * Y));
  float acc[CB];
#pragma unroll
  for (int c = 0; c < CB; ++c) acc[c] = (!TRANS && b && co0 + c < cout) ? b[co0 + c] : 0.f;
  const float *xn = x + (long long)n * cin * nvox;
  constexpr int KZ = D == 3 ? K : 1;
  for (int ci = 0; ci < cin; ++ci) {
    const float *xc = xn + (long long)ci * nvox;
    for (int dz = 0; dz < KZ; ++dz) {
      const int zz = D == 3 ? iz + dz - R : iz;
      if (zz < 0 || zz >= Z) continue;
      for (int dy = 0; dy < K; ++dy) {
        const int yy = iy + dy - R;
        if (yy < 0 || yy >= Y) continue;
        for (int dx = 0; dx < K; ++dx) {
          const int xx = ix + dx - R;
          if (xx < 0 || xx >= X) continue;
          const float v = xc[((long long)zz * Y + yy) * X + xx];
          const int tap = (dz * K + dy) * K + dx;
          const int taps = KZ * K * K;
#pragma unroll
          for (int c = 0; c < CB; ++c) {
            const int co = co0 + c;
            if (co >= cout) break;
            // forward: W[co][ci][tap]; transposed: W[ci'=co_out... ] mirrored
            long long wi;
            if (!TRANS) wi = ((long long)co * w_cin + ci) * taps + tap;
            else wi = ((long long)ci * w_cin + co) * taps + (taps - 1 - tap);
            acc[c] += __bfloat162float(w[wi]) * v;
          }
        }
      }
    }
  }
  float *yn = y + (long long)n * cout * nvox;
#pragma unroll
  for (int c = 0; c < CB; ++c) {
    const int co = co0 + c;
    if (co >= cout) break;
    float v = acc[c];
    if (relu && v < 0.f) v = 0.f;
    yn[(long long)co * nvox + t] = v;
  }
}

// weight gradient: dW[co][ci][tap] += sum_{n, p} dy[n, co, p] x[n, ci, p + tap - r]
// one block per (co, ci); threads stride over voxels, block-reduce per tap.
template <int D, int K>
__global__ void k_conv_wgrad(const float *__restrict__ x, const float *__restrict__ dy, float *__restrict__ dw,
                             float *__restrict__ db, int N, int cin, int cout, int X, int Y, int Z) {
  constexpr int R = K / 2, KZ = D == 3 ? K : 1, TAPS = KZ * K * K;
  const int co = blockIdx.x, ci = blockIdx.y;
  const long long nvox = (long long)X * Y * Z;
  float acc[TAPS];
#pragma unroll
  for (int q = 0; q < TAPS; ++q) acc[q] = 0.f;
  float accb = 0.f;
  for (int n = 0; n < N; ++n) {
    const float *g = dy + ((long long)n * cout + co) * nvox;
    const float *xc = x + ((long long)n * cin + ci) * nvox;
    for (long long t = threadIdx.x; t < nvox; t += blockDim.x) {
      const float gv = g[t];
      if (gv == 0.f) continue;
      const int ix = (int)(t % X), iy = (int)((t / X) % Y), iz = (int)(t / ((long long)X * Y));
      if (ci == 0) accb += gv;
#pragma unroll
      for (int dz = 0; dz < KZ; ++dz) {
        const int zz = D == 3 ? iz + dz - R : iz;
#pragma unroll
        for (int dyy = 0; dyy < K; ++dyy) {
          const int yy = iy + dyy - R;
#pragma unroll
          for (int dx = 0; dx < K; ++dx) {
            const int xx = ix + dx - R;
            const bool ok = xx >= 0 && xx < X && yy >= 0 && yy < Y && zz >= 0 && zz < Z;
            if (ok) acc[(dz * K + dyy) * K + dx] += gv * xc[((long long)zz * Y + yy) * X + xx];
          }
        }
      }
    }
  }
  __shared__ float red[NT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q <= TAPS; ++q) {
    float v = q < TAPS ? acc[q] : accb;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.f;
      for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) s += red[w2];
      if (q < TAPS) dw[((long long)co * cin + ci) * TAPS + q] += s;
      else if (ci == 0 && db) db[co] += s;
    }
  }
}

__global__ void k_scale(float *a, long long n, float s) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) a[t] *= s;
}

__global__ void k_relu_bwd(const float *a, float *g, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n && a[t] <= 0.f) g[t] = 0.f;
}

// average pool by 2 in every spatial dimension (sizes are even)
template <int D>
__global__ void k_pool(const float *x, float *y, long long NC, int X, int Y, int Z) {
  const int x2 = X / 2, y2 = Y / 2, z2 = D == 3 ? Z / 2 : 1;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long nv = (long long)x2 * y2 * z2;
  if (t >= NC * nv) return;
  long long c = t / nv, v = t % nv;
  int ix = (int)(v % x2), iy = (int)((v / x2) % y2), iz = (int)(v / ((long long)x2 * y2));
  const float *xc = x + c * (long long)X * Y * Z;
  float s = 0.f;
  for (int dz = 0; dz < (D == 3 ? 2 : 1); ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx)
        s += xc[((long long)(D == 3 ? 2 * iz + dz : 0) * Y + 2 * iy + dy) * X + 2 * ix + dx];
  y[t] = s * (D == 3 ? 0.125f : 0.25f);
}

template <int D>
__global__ void k_pool_bwd(const float *gy, float *gx, long long NC, int X, int Y, int Z) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long nv = (long long)X * Y * Z;
  if (t >= NC * nv) return;
  long long c = t / nv, v = t % nv;
  int ix = (int)(v % X), iy = (int)((v / X) % Y), iz = (int)(v / ((long long)X * Y));
  const int x2 = X / 2, y2 = Y / 2;
  const long long n2 = (long long)x2 * y2 * (D == 3 ? Z / 2 : 1);
  gx[t] = gy[c * n2 + ((long long)(D == 3 ? iz / 2 : 0) * y2 + iy / 2) * x2 + ix / 2] * (D == 3 ? 0.125f : 0.25f);
}

// nearest upsample by 2 into channel slot [c_off, c_off + C) of a wider tensor
template <int D>
__global__ void k_up(const float *x, float *y, int N, int C, int ctot, int c_off, int X, int Y, int Z) {
  // X, Y, Z: sizes of the (fine) output
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long nv = (long long)X * Y * Z;
  if (t >= (long long)N * C * nv) return;
  long long nc = t / nv, v = t % nv;
  int n = (int)(nc / C), c = (int)(nc % C);
  int ix = (int)(v % X), iy = (int)((v / X) % Y), iz = (int)(v / ((long long)X * Y));
  const int x2 = X / 2, y2 = Y / 2;
  const long long n2 = (long long)x2 * y2 * (D == 3 ? Z / 2 : 1);
  y[((long long)n * ctot + c_off + c) * nv + v] =
      x[((long long)n * C + c) * n2 + ((long long)(D == 3 ? iz / 2 : 0) * y2 + iy / 2) * x2 + ix / 2];
}

template <int D>
__global__ void k_up_bwd(const float *gy, float *gx, int N, int C, int ctot, int c_off, int X, int Y, int Z) {
  // gx: coarse (X/2...), gy: fine slot
  const int x2 = X / 2, y2 = Y / 2, z2 = D == 3 ? Z / 2 : 1;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n2 = (long long)x2 * y2 * z2, nv = (long long)X * Y * Z;
  if (t >= (long long)N * C * n2) return;
  long long nc = t / n2, v = t % n2;
  int n = (int)(nc / C), c = (int)(nc % C);
  int ix = (int)(v % x2), iy = (int)((v / x2) % y2), iz = (int)(v / ((long long)x2 * y2));
  const float *g = gy + ((long long)n * ctot + c_off + c) * nv;
  float s = 0.f;
  for (int dz = 0; dz < (D == 3 ? 2 : 1); ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx)
        s += g[((long long)(D == 3 ? 2 * iz + dz : 0) * Y + 2 * iy + dy) * X + 2 * ix + dx];
  gx[t] = s;
}

// copy channels [0, C) of a tensor into slot [c_off, c_off + C) of a wider one (and back)
__global__ void k_slot_copy(const float *src, float *dst, int N, int C, int csrc, int soff, int cdst, int doff,
                            long long nv, int accumulate) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * C * nv) return;
  long long nc = t / nv, v = t % nv;
  int n = (int)(nc / C), c = (int)(nc % C);
  float val = src[((long long)n * csrc + soff + c) * nv + v];
  float *d = dst + ((long long)n * cdst + doff + c) * nv + v;
  if (accumulate) *d += val; else *d = val;
}

// MSE loss between y and target (both N x C x nv): grad = 2 (y - t) / count.
// The loss is summed in a fixed order so that it is the same bit for bit on
// every call: a fixed grid of MSE_BLOCKS blocks strides over the elements,
// each block reduces its threads' sums in a fixed tree into partial[block],
// and k_mse_final adds the partials in a fixed tree.
constexpr int MSE_BLOCKS = 256;

__device__ __forceinline__ double block_sum_fixed(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) s += sh[w2];
  return s;
}

// With an output scale s (y = s h), the loss is taken in units of s,
// mean(((y - t) / s)^2), and g receives its gradient with respect to the
// head's output h: 2 (y - t) / (s n).  inv_s = 1 / s (1 for s = 0 or 1).
__global__ void k_mse(const float *y, const float *t, float *g, long long n, double *partial, float inv_s) {
  __shared__ double sh[NT / 32];
  double d2 = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = (y[i] - t[i]) * inv_s;
    g[i] = 2.f * d / (float)n;
    d2 += (double)d * d;
  }
  const double s = block_sum_fixed(d2, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_mse_final(const double *partial, long long n, double *loss) {
  __shared__ double sh[NT / 32];
  const double s = block_sum_fixed(threadIdx.x < MSE_BLOCKS ? partial[threadIdx.x] : 0.0, sh);
  if (threadIdx.x == 0) *loss = s / (double)n;
}

// Adam's denominator guard: far below any gradient the losses here produce
// (means over millions of voxels make per-parameter gradients of 1e-9 and
// less), so that the update stays scale-free
#ifndef EP_ADAM_EPS
#define EP_ADAM_EPS 1e-15f
#endif
constexpr float ADAM_EPS = EP_ADAM_EPS;

__global__ void k_adam(float *w, __nv_bfloat16 *wb, const float *g, float *m, float *v, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(const float *w, __nv_bfloat16 *wb, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

}  // namespace

// ----------------------------------------------------------------------------
struct Layer {
  int cin, cout, k;
  long long woff, boff;   // offsets into the parameter vector
};

struct UNet {
  int D, cin, cout, base, levels;
  std::vector<Layer> layers;  // enc (2 per level), dec (2 per level except last), head
  long long nparam = 0;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *wb = nullptr;
  long long step = 0;
  // activations for the current shape
  int N = 0, X = 0, Y = 0, Z = 0;
  std::vector<float *> act, grad;   // per stored tensor
  std::vector<int> act_c;           // channels of each stored tensor
  std::vector<int> act_lvl;         // level (resolution) of each stored tensor
  float *scratch = nullptr, *scratch2 = nullptr;
  long long scratch_n = 0;
  double *dloss = nullptr;
  cudaStream_t st = nullptr;
  // tensor-core inference: weights packed per layer in the MMA operand
  // layout (offset -1: the layer runs on CUDA cores), the channels-last BF16
  // copy of a layer's input, and the kernels' error word
  __nv_bfloat16 *wpk = nullptr;
  std::vector<long long> pk_off;
  __nv_bfloat16 *xcl = nullptr;
  long long xcl_n = 0;
  int *terr = nullptr;
  // the network's output is out_scale times the head's: training on targets
  // of any magnitude keeps the head's values of order one
  float out_scale = 1.f;
};

static long long vox(const UNet &u, int lvl) {
  long long s = 1;
  s *= (u.X >> lvl);
  s *= (u.Y >> lvl);
  if (u.D == 3) s *= (u.Z >> lvl);
  return s;
}

// Build the layer table and parameter offsets.
static void unet_layers(UNet &u) {
  long long off = 0;
  auto add = [&](int ci, int co, int k) {
    Layer L{ci, co, k, off, 0};
    long long taps = (long long)k * k * (u.D == 3 ? k : 1);
    off += (long long)ci * co * taps;
    L.boff = off;
    off += co;
    u.layers.push_back(L);
  };
  int c_prev = u.cin;
  for (int l = 0; l < u.levels; ++l) {
    int c = u.base << l;
    add(c_prev, c, 3);
    add(c, c, 3);
    c_prev = c;
  }
  for (int l = u.levels - 2; l >= 0; --l) {
    int c = u.base << l, cup = u.base << (l + 1);
    add(cup + c, c, 3);
    add(c, c, 3);
  }
  add(u.base, u.cout, 1);
  u.nparam = off;
}

// offsets of the packed tensor-core weights per layer (-1: CUDA cores); total
// BF16 elements
static long long tc_layout(UNet &u) {
  long long off = 0;
  u.pk_off.assign(u.layers.size(), -1);
  for (size_t q = 0; q < u.layers.size(); ++q) {
    const Layer &L = u.layers[q];
    if (!conv_tc_supported(L.k, L.cout)) continue;
    u.pk_off[q] = off;
    const long long taps = u.D == 3 ? 27 : 9;
    off += taps * conv_tc_cinp(L.cin) * L.cout;
  }
  return off;
}

// repack the BF16 weights for the tensor cores (after every weight change)
static void tc_pack(UNet &u) {
  for (size_t q = 0; q < u.layers.size(); ++q) {
    if (u.pk_off[q] < 0) continue;
    const Layer &L = u.layers[q];
    conv_tc_pack_weights(u.wb + L.woff, L.cin, L.cout, u.D == 3 ? 27 : 9, u.wpk + u.pk_off[q], u.st);
  }
}

// BF16 elements of the largest channels-last layer input at shape (N, X, Y, Z)
static long long tc_xcl_elems(const UNet &u, int N, int X, int Y, int Z) {
  long long best = 0;
  int li = 0;
  auto lvl_vox = [&](int l) {
    long long v = (long long)(X >> l) * (Y >> l);
    return u.D == 3 ? v * (Z >> l) : v;
  };
  for (int l = 0; l < u.levels; ++l)
    for (int r = 0; r < 2; ++r, ++li)
      if (u.pk_off[li] >= 0) best = std::max(best, (long long)N * lvl_vox(l) * conv_tc_cinp(u.layers[li].cin));
  for (int l = u.levels - 2; l >= 0; --l)
    for (int r = 0; r < 2; ++r, ++li)
      if (u.pk_off[li] >= 0) best = std::max(best, (long long)N * lvl_vox(l) * conv_tc_cinp(u.layers[li].cin));
  return best;
}

}  // namespace ep

namespace ep {

static cudaError_t ensure_shape(UNet &u, int N, int X, int Y, int Z) {
  if (u.N == N && u.X == X && u.Y == Y && u.Z == Z) return cudaSuccess;
  for (float *p : u.act) cudaFree(p);
  for (float *p : u.grad) cudaFree(p);
  u.act.clear(); u.grad.clear(); u.act_c.clear(); u.act_lvl.clear();
  if (u.scratch) cudaFree(u.scratch);
  if (u.scratch2) cudaFree(u.scratch2);
  u.scratch = u.scratch2 = nullptr;
  u.N = N; u.X = X; u.Y = Y; u.Z = Z;
  // tensors in forward order: e[l][0], e[l][1], pool[l] (l < L-1), then per
  // decoder level: cat, d0, d1; then the head output
  auto add = [&](int c, int lvl) {
    float *a = nullptr, *g = nullptr;
    size_t bytes = (size_t)N * c * vox(u, lvl) * sizeof(float);
    cudaError_t e = cudaMalloc((void **)&a, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&g, bytes);
    u.act.push_back(a); u.grad.push_back(g); u.act_c.push_back(c); u.act_lvl.push_back(lvl);
    return e;
  };
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < u.levels && e == cudaSuccess; ++l) {
    int c = u.base << l;
    e = add(c, l);
    if (e == cudaSuccess) e = add(c, l);
    if (e == cudaSuccess && l < u.levels - 1) e = add(c, l + 1);
  }
  for (int l = u.levels - 2; l >= 0 && e == cudaSuccess; --l) {
    int c = u.base << l, cup = u.base << (l + 1);
    e = add(cup + c, l);
    if (e == cudaSuccess) e = add(c, l);
    if (e == cudaSuccess) e = add(c, l);
  }
  if (e == cudaSuccess) e = add(u.cout, 0);
  long long big = (long long)N * (u.base << (u.levels - 1)) * 2 * vox(u, 0);
  if (e == cudaSuccess) e = cudaMalloc((void **)&u.scratch, big * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void **)&u.scratch2, big * sizeof(float));
  u.scratch_n = big;
  if (u.xcl) cudaFree(u.xcl);
  u.xcl = nullptr;
  u.xcl_n = tc_xcl_elems(u, N, X, Y, Z);
  if (e == cudaSuccess && u.xcl_n > 0) e = cudaMalloc((void **)&u.xcl, u.xcl_n * sizeof(__nv_bfloat16));
  return e;
}

// tensor indices of the forward graph
struct Idx {
  int e0[8], e1[8], pool[8], cat[8], d0[8], d1[8], out;
};
static Idx indices(const UNet &u) {
  Idx I{};
  int q = 0;
  for (int l = 0; l < u.levels; ++l) {
    I.e0[l] = q++;
    I.e1[l] = q++;
    if (l < u.levels - 1) I.pool[l] = q++;
  }
  for (int l = u.levels - 2; l >= 0; --l) {
    I.cat[l] = q++;
    I.d0[l] = q++;
    I.d1[l] = q++;
  }
  I.out = q++;
  return I;
}

// one convolution on the tensor cores: the input to channels-last BF16, then
// the implicit GEMM (the caller has checked that the layer is supported)
template <int D>
static void conv_tc(const UNet &u, int li, int N, int X, int Y, int Z, const float *x, float *y, int relu,
                    __nv_bfloat16 *xcl) {
  const Layer &L = u.layers[li];
  const long long nv = (long long)X * Y * Z;
  conv_tc_to_channels_last(x, N, L.cin, nv, conv_tc_cinp(L.cin), xcl, u.st);
  conv_tc_forward(D, xcl, N, X, Y, Z, L.cin, u.wpk + u.pk_off[li], u.w + L.boff, L.cout, relu, y, u.terr, u.st);
}

template <int D>
static void conv_fwd(UNet &u, const Layer &L, const float *x, float *y, int lvl, int relu, bool tc = false) {
  const long long nv = vox(u, lvl);
  const int li = (int)(&L - u.layers.data());
  if (tc && u.pk_off[li] >= 0) {
    conv_tc<D>(u, li, u.N, u.X >> lvl, u.Y >> lvl, D == 3 ? (u.Z >> lvl) : 1, x, y, relu, u.xcl);
    return;
  }
  dim3 grid(nblk(nv), (L.cout + 7) / 8, u.N);
  const int X = u.X >> lvl, Y = u.Y >> lvl, Z = D == 3 ? (u.Z >> lvl) : 1;
  if (L.k == 3)
    k_conv<D, 3, false><<<grid, NT, 0, u.st>>>(x, u.wb + L.woff, u.w + L.boff, y, u.N, L.cin, L.cout, X, Y, Z, relu,
                                               L.cin, L.cout);
  else
    k_conv<D, 1, false><<<grid, NT, 0, u.st>>>(x, u.wb + L.woff, u.w + L.boff, y, u.N, L.cin, L.cout, X, Y, Z, relu,
                                               L.cin, L.cout);
}

// data gradient gx (cin channels) from gy (cout channels); weight gradient into u.g
template <int D>
static void conv_bwd(UNet &u, const Layer &L, const float *x, const float *gy, float *gx, int lvl) {
  const long long nv = vox(u, lvl);
  const int X = u.X >> lvl, Y = u.Y >> lvl, Z = D == 3 ? (u.Z >> lvl) : 1;
  dim3 wg(L.cout, L.cin);
  if (L.k == 3) k_conv_wgrad<D, 3><<<wg, NT, 0, u.st>>>(x, gy, u.g + L.woff, u.g + L.boff, u.N, L.cin, L.cout, X, Y, Z);
  else k_conv_wgrad<D, 1><<<wg, NT, 0, u.st>>>(x, gy, u.g + L.woff, u.g + L.boff, u.N, L.cin, L.cout, X, Y, Z);
  if (!gx) return;
  dim3 grid(nblk(nv), (L.cin + 7) / 8, u.N);
  if (L.k == 3)
    k_conv<D, 3, true><<<grid, NT, 0, u.st>>>(gy, u.wb + L.woff, nullptr, gx, u.N, L.cout, L.cin, X, Y, Z, 0, L.cin,
                                              L.cout);
  else
    k_conv<D, 1, true><<<grid, NT, 0, u.st>>>(gy, u.wb + L.woff, nullptr, gx, u.N, L.cout, L.cin, X, Y, Z, 0, L.cin,
                                              L.cout);
}

static void relu_bwd(UNet &u, int q) {
  long long n = (long long)u.N * u.act_c[q] * vox(u, u.act_lvl[q]);
  k_relu_bwd<<<nblk(n), NT, 0, u.st>>>(u.act[q], u.grad[q], n);
}

template <int D>
static void forward(UNet &u, const float *x, bool tc = false) {
  const Idx I = indices(u);
  int li = 0;
  const float *in = x;
  for (int l = 0; l < u.levels; ++l) {
    conv_fwd<D>(u, u.layers[li++], in, u.act[I.e0[l]], l, 1, tc);
    conv_fwd<D>(u, u.layers[li++], u.act[I.e0[l]], u.act[I.e1[l]], l, 1, tc);
    if (l < u.levels - 1) {
      const int X = u.X >> l, Y = u.Y >> l, Z = D == 3 ? (u.Z >> l) : 1;
      long long n = (long long)u.N * u.act_c[I.pool[l]] * vox(u, l + 1);
      k_pool<D><<<nblk(n), NT, 0, u.st>>>(u.act[I.e1[l]], u.act[I.pool[l]], (long long)u.N * (u.base << l), X, Y, Z);
      in = u.act[I.pool[l]];
    }
  }
  const float *prev = u.act[I.e1[u.levels - 1]];
  for (int l = u.levels - 2; l >= 0; --l) {
    const int c = u.base << l, cup = u.base << (l + 1);
    const int X = u.X >> l, Y = u.Y >> l, Z = D == 3 ? (u.Z >> l) : 1;
    const long long nv = vox(u, l);
    k_up<D><<<nblk((long long)u.N * cup * nv), NT, 0, u.st>>>(prev, u.act[I.cat[l]], u.N, cup, cup + c, 0, X, Y, Z);
    k_slot_copy<<<nblk((long long)u.N * c * nv), NT, 0, u.st>>>(u.act[I.e1[l]], u.act[I.cat[l]], u.N, c, c, 0,
                                                                cup + c, cup, nv, 0);
    conv_fwd<D>(u, u.layers[li++], u.act[I.cat[l]], u.act[I.d0[l]], l, 1, tc);
    conv_fwd<D>(u, u.layers[li++], u.act[I.d0[l]], u.act[I.d1[l]], l, 1, tc);
    prev = u.act[I.d1[l]];
  }
  conv_fwd<D>(u, u.layers[li++], prev, u.act[I.out], 0, 0);
  if (u.out_scale != 1.f) {
    const long long no = (long long)u.N * u.cout * vox(u, 0);
    k_scale<<<nblk(no), NT, 0, u.st>>>(u.act[I.out], no, u.out_scale);
  }
}

// gradients of all parameters given d loss / d out in u.grad[out]
template <int D>
static void backward(UNet &u, const float *x) {
  const Idx I = indices(u);
  const int nl = (int)u.layers.size();
  int li = nl - 1;
  // zero the activation gradients that are accumulated into: every e1 (skip
  // and pool/up paths) and the decoder outputs below the finest level (their
  // only contribution arrives through the upsampling of the next finer level)
  for (int l = 0; l < u.levels; ++l) {
    long long n = (long long)u.N * u.act_c[I.e1[l]] * vox(u, l);
    cudaMemsetAsync(u.grad[I.e1[l]], 0, n * sizeof(float), u.st);
  }
  for (int l = 1; l <= u.levels - 2; ++l) {
    long long n = (long long)u.N * u.act_c[I.d1[l]] * vox(u, l);
    cudaMemsetAsync(u.grad[I.d1[l]], 0, n * sizeof(float), u.st);
  }
  const int top = u.levels == 1 ? I.e1[0] : I.d1[0];
  // head
  {
    long long n = (long long)u.N * u.base * vox(u, 0);
    if (u.levels == 1) {
      conv_bwd<D>(u, u.layers[li--], u.act[top], u.grad[I.out], u.scratch, 0);
      k_slot_copy<<<nblk(n), NT, 0, u.st>>>(u.scratch, u.grad[top], u.N, u.base, u.base, 0, u.base, 0, vox(u, 0), 1);
    } else {
      conv_bwd<D>(u, u.layers[li--], u.act[top], u.grad[I.out], u.grad[top], 0);
    }
  }
  // decoder, finest level first
  for (int l = 0; l <= u.levels - 2; ++l) {
    const int c = u.base << l, cup = u.base << (l + 1);
    const int X = u.X >> l, Y = u.Y >> l, Z = D == 3 ? (u.Z >> l) : 1;
    const long long nv = vox(u, l);
    const Layer &L1 = u.layers[li--];
    const Layer &L0 = u.layers[li--];
    relu_bwd(u, I.d1[l]);
    conv_bwd<D>(u, L1, u.act[I.d0[l]], u.grad[I.d1[l]], u.grad[I.d0[l]], l);
    relu_bwd(u, I.d0[l]);
    conv_bwd<D>(u, L0, u.act[I.cat[l]], u.grad[I.d0[l]], u.grad[I.cat[l]], l);
    // split the concatenation: upsampled part -> coarser tensor, skip -> e1[l]
    k_slot_copy<<<nblk((long long)u.N * c * nv), NT, 0, u.st>>>(u.grad[I.cat[l]], u.grad[I.e1[l]], u.N, c, cup + c,
                                                                cup, c, 0, nv, 1);
    const int coarse = l + 1 == u.levels - 1 ? I.e1[l + 1] : I.d1[l + 1];
    const long long n2 = (long long)u.N * cup * vox(u, l + 1);
    k_up_bwd<D><<<nblk(n2), NT, 0, u.st>>>(u.grad[I.cat[l]], u.scratch, u.N, cup, cup + c, 0, X, Y, Z);
    k_slot_copy<<<nblk(n2), NT, 0, u.st>>>(u.scratch, u.grad[coarse], u.N, cup, cup, 0, cup, 0, vox(u, l + 1), 1);
  }
  // encoder, coarsest level first
  for (int l = u.levels - 1; l >= 0; --l) {
    const Layer &L1 = u.layers[2 * l + 1];
    const Layer &L0 = u.layers[2 * l];
    relu_bwd(u, I.e1[l]);
    conv_bwd<D>(u, L1, u.act[I.e0[l]], u.grad[I.e1[l]], u.grad[I.e0[l]], l);
    relu_bwd(u, I.e0[l]);
    const float *in = l == 0 ? x : u.act[I.pool[l - 1]];
    float *gin = l == 0 ? nullptr : u.grad[I.pool[l - 1]];
    conv_bwd<D>(u, L0, in, u.grad[I.e0[l]], gin, l);
    if (l > 0) {
      const int X = u.X >> (l - 1), Y = u.Y >> (l - 1), Z = D == 3 ? (u.Z >> (l - 1)) : 1;
      const int cl = u.base << (l - 1);
      long long n = (long long)u.N * cl * vox(u, l - 1);
      k_pool_bwd<D><<<nblk(n), NT, 0, u.st>>>(u.grad[I.pool[l - 1]], u.scratch, (long long)u.N * cl, X, Y, Z);
      k_slot_copy<<<nblk(n), NT, 0, u.st>>>(u.scratch, u.grad[I.e1[l - 1]], u.N, cl, cl, 0, cl, 0, vox(u, l - 1), 1);
    }
  }
}

}  // namespace ep

// ============================================================================
using namespace ep;

struct ep_net {
  UNet u;
  std::string err;
};

static thread_local std::string g_net_err;

static ep_status nfail(ep_net *n, ep_status st, const std::string &m) {
  if (n) n->err = m;
  g_net_err = m;
  return st;
}

#define NCK(n, call)                                                                                  \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return nfail((n), EP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// the tensor-core kernels' error word: a bounded wait that ran out
static ep_status tc_status(ep_net *n) {
  int e = 0;
  NCK(n, cudaMemcpyAsync(&e, n->u.terr, sizeof(int), cudaMemcpyDeviceToHost, n->u.st));
  NCK(n, cudaStreamSynchronize(n->u.st));
  if (e) {
    cudaMemsetAsync(n->u.terr, 0, sizeof(int), n->u.st);
    return nfail(n, EP_ERR_TIMEOUT, "tensor-core convolution: a bounded wait gave up");
  }
  return EP_OK;
}

static bool shape_ok(const ep_net *n, const int size[3]) {
  const int m = 1 << (n->u.levels - 1);
  for (int d = 0; d < n->u.D; ++d)
    if (size[d] < m || size[d] % m) return false;
  return true;
}

// ---- forward pass that allocates nothing ----------------------------------
// ep_net_forward_static keeps its activations in one file-scope device array
// instead of buffers sized on first use.  It exists for callers that must not
// allocate device memory while they run: a solver loop that applies the warm
// start between load increments on a device whose memory is already spoken
// for (the grid's arena and the caller's own allocator pool can hold almost
// all of it, so a new cudaMalloc may fail), and latency-bound loops, because
// cudaMalloc and cudaFree synchronise the whole device and stall every other
// stream.  The array holds EP_NET_STATIC_FLOATS floats; larger shapes are
// rejected.  Every call on a device shares it, so calls whose kernels overlap
// on the GPU (different streams without ordering between them) race.  None of
// it has to start at zero: each activation is written in full before it is
// read.  The first call on a device looks up the array's address (with that
// device current); make that first call before any stream capture.
static __device__ __align__(256) float g_static_act[EP_NET_STATIC_FLOATS];

static std::mutex g_static_mu;
static float *g_static_ptr[64];

// device address of g_static_act on the current device (set up once)
static ep_status static_act(ep_net *n, float **out) {
  int dev = 0;
  NCK(n, cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return nfail(n, EP_ERR_ARG, "ep_net_forward_static: device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    NCK(n, cudaGetSymbolAddress(&p, g_static_act));
    g_static_ptr[dev] = (float *)p;
  }
  *out = g_static_ptr[dev];
  return EP_OK;
}

struct Shp {
  int N, X, Y, Z;
};

static long long svox(const UNet &u, const Shp &s, int lvl) {
  long long v = (long long)(s.X >> lvl) * (s.Y >> lvl);
  if (u.D == 3) v *= (s.Z >> lvl);
  return v;
}

// floats the forward's activations take at shape s, with each tensor's
// offset (in the order of indices()) when off is non-null
static long long static_layout(const UNet &u, const Shp &s, long long *off) {
  long long total = 0;
  int q = 0;
  auto add = [&](int c, int lvl) {
    if (off) off[q] = total;
    ++q;
    total += ((long long)s.N * c * svox(u, s, lvl) + 63) / 64 * 64;  // 256-byte aligned tensors
  };
  for (int l = 0; l < u.levels; ++l) {
    const int c = u.base << l;
    add(c, l);
    add(c, l);
    if (l < u.levels - 1) add(c, l + 1);
  }
  for (int l = u.levels - 2; l >= 0; --l) {
    const int c = u.base << l, cup = u.base << (l + 1);
    add(cup + c, l);
    add(c, l);
    add(c, l);
  }
  // the channels-last BF16 input of the tensor-core convolutions (two per
  // float), at the index of the head output (which is written to y)
  if (off) off[q] = total;
  total += (tc_xcl_elems(u, s.N, s.X, s.Y, s.Z) / 2 + 64) / 64 * 64;
  return total;
}

template <int D>
static void conv_fwd_s(const UNet &u, const Shp &s, const Layer &L, const float *x, float *y, int lvl, int relu,
                       __nv_bfloat16 *xcl) {
  const long long nv = svox(u, s, lvl);
  const int li = (int)(&L - u.layers.data());
  if (u.pk_off[li] >= 0) {
    conv_tc<D>(u, li, s.N, s.X >> lvl, s.Y >> lvl, D == 3 ? (s.Z >> lvl) : 1, x, y, relu, xcl);
    return;
  }
  dim3 grid(nblk(nv), (L.cout + 7) / 8, s.N);
  const int X = s.X >> lvl, Y = s.Y >> lvl, Z = D == 3 ? (s.Z >> lvl) : 1;
  if (L.k == 3)
    k_conv<D, 3, false><<<grid, NT, 0, u.st>>>(x, u.wb + L.woff, u.w + L.boff, y, s.N, L.cin, L.cout, X, Y, Z, relu,
                                               L.cin, L.cout);
  else
    k_conv<D, 1, false><<<grid, NT, 0, u.st>>>(x, u.wb + L.woff, u.w + L.boff, y, s.N, L.cin, L.cout, X, Y, Z, relu,
                                               L.cin, L.cout);
}

// the network's forward pass with activations at act + off[q] and the head
// writing straight into y; same kernels and launch shapes as forward()
template <int D>
static void forward_static(const UNet &u, const Shp &s, const float *x, float *act, const long long *off, float *y) {
  const Idx I = indices(u);
  __nv_bfloat16 *xcl = reinterpret_cast<__nv_bfloat16 *>(act + off[I.out]);
  int li = 0;
  const float *in = x;
  for (int l = 0; l < u.levels; ++l) {
    conv_fwd_s<D>(u, s, u.layers[li++], in, act + off[I.e0[l]], l, 1, xcl);
    conv_fwd_s<D>(u, s, u.layers[li++], act + off[I.e0[l]], act + off[I.e1[l]], l, 1, xcl);
    if (l < u.levels - 1) {
      const int X = s.X >> l, Y = s.Y >> l, Z = D == 3 ? (s.Z >> l) : 1;
      const long long n = (long long)s.N * (u.base << l) * svox(u, s, l + 1);
      k_pool<D><<<nblk(n), NT, 0, u.st>>>(act + off[I.e1[l]], act + off[I.pool[l]], (long long)s.N * (u.base << l),
                                          X, Y, Z);
      in = act + off[I.pool[l]];
    }
  }
  const float *prev = act + off[I.e1[u.levels - 1]];
  for (int l = u.levels - 2; l >= 0; --l) {
    const int c = u.base << l, cup = u.base << (l + 1);
    const int X = s.X >> l, Y = s.Y >> l, Z = D == 3 ? (s.Z >> l) : 1;
    const long long nv = svox(u, s, l);
    float *cat = act + off[I.cat[l]];
    k_up<D><<<nblk((long long)s.N * cup * nv), NT, 0, u.st>>>(prev, cat, s.N, cup, cup + c, 0, X, Y, Z);
    k_slot_copy<<<nblk((long long)s.N * c * nv), NT, 0, u.st>>>(act + off[I.e1[l]], cat, s.N, c, c, 0, cup + c, cup,
                                                                nv, 0);
    conv_fwd_s<D>(u, s, u.layers[li++], cat, act + off[I.d0[l]], l, 1, xcl);
    conv_fwd_s<D>(u, s, u.layers[li++], act + off[I.d0[l]], act + off[I.d1[l]], l, 1, xcl);
    prev = act + off[I.d1[l]];
  }
  conv_fwd_s<D>(u, s, u.layers[li++], prev, y, 0, 0, xcl);
  if (u.out_scale != 1.f) {
    const long long no = (long long)s.N * u.cout * svox(u, s, 0);
    k_scale<<<nblk(no), NT, 0, u.st>>>(y, no, u.out_scale);
  }
}

extern "C" {

ep_status ep_net_create(int ndim, int in_ch, int out_ch, int base, int levels, unsigned long long seed, void *stream,
                        ep_net **out) {
  if (!out || (ndim != 2 && ndim != 3) || in_ch < 1 || out_ch < 1 || base < 1 || levels < 1 || levels > 6)
    return nfail(nullptr, EP_ERR_ARG, "ep_net_create: bad arguments");
  ep_net *n = new ep_net();
  UNet &u = n->u;
  u.D = ndim; u.cin = in_ch; u.cout = out_ch; u.base = base; u.levels = levels;
  u.st = (cudaStream_t)stream;
  unet_layers(u);
  // He-uniform initialisation from splitmix64 (seeded); biases and the head zero
  std::vector<float> w(u.nparam, 0.f);
  unsigned long long st = seed;
  auto rnd = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    unsigned long long z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  for (size_t li = 0; li + 1 < u.layers.size(); ++li) {
    const Layer &L = u.layers[li];
    long long taps = (long long)L.k * L.k * (ndim == 3 ? L.k : 1);
    double bound = sqrt(6.0 / (double)(L.cin * taps));
    for (long long q = 0; q < (long long)L.cin * L.cout * taps; ++q) w[L.woff + q] = (float)((2.0 * rnd() - 1.0) * bound);
  }
  const long long np = u.nparam;
  if (cudaMalloc((void **)&u.w, np * 4) != cudaSuccess || cudaMalloc((void **)&u.g, np * 4) != cudaSuccess ||
      cudaMalloc((void **)&u.m, np * 4) != cudaSuccess || cudaMalloc((void **)&u.v, np * 4) != cudaSuccess ||
      cudaMalloc((void **)&u.wb, np * 2) != cudaSuccess || cudaMalloc((void **)&u.dloss, 8 * (1 + MSE_BLOCKS)) != cudaSuccess) {
    ep_net_destroy(n);
    return nfail(nullptr, EP_ERR_OOM, "ep_net_create: allocation failed");
  }
  const long long npk = tc_layout(u);
  if ((npk > 0 && cudaMalloc((void **)&u.wpk, npk * sizeof(__nv_bfloat16)) != cudaSuccess) ||
      cudaMalloc((void **)&u.terr, sizeof(int)) != cudaSuccess) {
    ep_net_destroy(n);
    return nfail(nullptr, EP_ERR_OOM, "ep_net_create: allocation failed");
  }
  cudaMemset(u.terr, 0, sizeof(int));
  cudaMemcpy(u.w, w.data(), np * 4, cudaMemcpyHostToDevice);
  cudaMemset(u.m, 0, np * 4);
  cudaMemset(u.v, 0, np * 4);
  k_to_bf16<<<nblk(np), NT, 0, u.st>>>(u.w, u.wb, np);
  tc_pack(u);
  if (cudaStreamSynchronize(u.st) != cudaSuccess) {
    ep_net_destroy(n);
    return nfail(nullptr, EP_ERR_CUDA, "ep_net_create: initialisation failed");
  }
  *out = n;
  return EP_OK;
}

ep_status ep_net_param_count(ep_net *n, long long *count) {
  if (!n || !count) return nfail(n, EP_ERR_ARG, "null argument");
  *count = n->u.nparam;
  return EP_OK;
}

ep_status ep_net_get_params(ep_net *n, float *host, long long count) {
  if (!n || !host || count != n->u.nparam) return nfail(n, EP_ERR_ARG, "ep_net_get_params: bad arguments");
  NCK(n, cudaMemcpy(host, n->u.w, count * 4, cudaMemcpyDeviceToHost));
  return EP_OK;
}

ep_status ep_net_set_params(ep_net *n, const float *host, long long count) {
  if (!n || !host || count != n->u.nparam) return nfail(n, EP_ERR_ARG, "ep_net_set_params: bad arguments");
  NCK(n, cudaMemcpy(n->u.w, host, count * 4, cudaMemcpyHostToDevice));
  k_to_bf16<<<nblk(count), NT, 0, n->u.st>>>(n->u.w, n->u.wb, count);
  tc_pack(n->u);
  NCK(n, cudaStreamSynchronize(n->u.st));
  return EP_OK;
}

ep_status ep_net_forward(ep_net *n, const float *x, int N, const int size[3], float *y) {
  if (!n || !x || !y || N < 1 || !size || !shape_ok(n, size))
    return nfail(n, EP_ERR_ARG, "ep_net_forward: sizes must be multiples of 2^(levels-1)");
  UNet &u = n->u;
  NCK(n, ensure_shape(u, N, size[0], size[1], u.D == 3 ? size[2] : 1));
  if (u.D == 2) forward<2>(u, x, true); else forward<3>(u, x, true);
  const long long no = (long long)N * u.cout * vox(u, 0);
  NCK(n, cudaMemcpyAsync(y, u.act[indices(u).out], no * 4, cudaMemcpyDeviceToDevice, u.st));
  NCK(n, cudaGetLastError());
  return tc_status(n);
}

// See the declaration in ep.h and the notes above g_static_act.
ep_status ep_net_forward_static(ep_net *n, const float *x, int N, const int size[3], float *y) {
  if (!n || !x || !y || N < 1 || !size || !shape_ok(n, size))
    return nfail(n, EP_ERR_ARG, "ep_net_forward_static: sizes must be multiples of 2^(levels-1)");
  const UNet &u = n->u;
  const Shp s{N, size[0], size[1], u.D == 3 ? size[2] : 1};
  long long off[64];
  const long long need = static_layout(u, s, off);
  if (need > EP_NET_STATIC_FLOATS)
    return nfail(n, EP_ERR_ARG,
                 "ep_net_forward_static: this shape needs " + std::to_string(need) +
                     " floats of activations, above the static limit of " +
                     std::to_string((long long)EP_NET_STATIC_FLOATS) + " (use ep_net_forward)");
  float *act = nullptr;
  const ep_status r = static_act(n, &act);
  if (r != EP_OK) return r;
  if (u.D == 2) forward_static<2>(u, s, x, act, off, y);
  else forward_static<3>(u, s, x, act, off, y);
  NCK(n, cudaGetLastError());
  return tc_status(n);
}

static ep_status net_grads(ep_net *n, const float *x, const float *t, int N, const int size[3], double *loss) {
  UNet &u = n->u;
  NCK(n, ensure_shape(u, N, size[0], size[1], u.D == 3 ? size[2] : 1));
  if (u.D == 2) forward<2>(u, x); else forward<3>(u, x);
  const Idx I = indices(u);
  const long long no = (long long)N * u.cout * vox(u, 0);
  NCK(n, cudaMemsetAsync(u.g, 0, u.nparam * 4, u.st));
  const float inv_s = u.out_scale > 0.f ? 1.f / u.out_scale : 1.f;
  k_mse<<<MSE_BLOCKS, NT, 0, u.st>>>(u.act[I.out], t, u.grad[I.out], no, u.dloss + 1, inv_s);
  k_mse_final<<<1, NT, 0, u.st>>>(u.dloss + 1, no, u.dloss);
  if (u.D == 2) backward<2>(u, x); else backward<3>(u, x);
  NCK(n, cudaGetLastError());
  if (loss) NCK(n, cudaMemcpyAsync(loss, u.dloss, 8, cudaMemcpyDeviceToHost, u.st));
  NCK(n, cudaStreamSynchronize(u.st));
  return EP_OK;
}

ep_status ep_net_gradients(ep_net *n, const float *x, const float *t, int N, const int size[3], double *loss,
                           float *grad_host, long long count) {
  if (!n || !x || !t || N < 1 || !size || !shape_ok(n, size) || (grad_host && count != n->u.nparam))
    return nfail(n, EP_ERR_ARG, "ep_net_gradients: bad arguments");
  ep_status r = net_grads(n, x, t, N, size, loss);
  if (r != EP_OK) return r;
  if (grad_host) NCK(n, cudaMemcpy(grad_host, n->u.g, count * 4, cudaMemcpyDeviceToHost));
  return EP_OK;
}

ep_status ep_net_train_step(ep_net *n, const float *x, const float *t, int N, const int size[3], float lr,
                            double *loss) {
  if (!n || !x || !t || N < 1 || !size || !shape_ok(n, size) || !(lr > 0.f))
    return nfail(n, EP_ERR_ARG, "ep_net_train_step: bad arguments");
  ep_status r = net_grads(n, x, t, N, size, loss);
  if (r != EP_OK) return r;
  UNet &u = n->u;
  u.step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)u.step), c2 = 1.f - powf(b2, (float)u.step);
  k_adam<<<nblk(u.nparam), NT, 0, u.st>>>(u.w, u.wb, u.g, u.m, u.v, u.nparam, lr, b1, b2, ADAM_EPS, c1, c2);
  tc_pack(u);
  NCK(n, cudaGetLastError());
  NCK(n, cudaStreamSynchronize(u.st));
  return EP_OK;
}

ep_status ep_net_set_output_scale(ep_net *n, double scale) {
  if (!n || !(scale >= 0.0) || !std::isfinite(scale))
    return nfail(n, EP_ERR_ARG, "ep_net_set_output_scale: need a finite scale >= 0");
  n->u.out_scale = (float)scale;
  return EP_OK;
}

ep_status ep_net_get_output_scale(ep_net *n, double *scale) {
  if (!n || !scale) return nfail(n, EP_ERR_ARG, "ep_net_get_output_scale: null argument");
  *scale = n->u.out_scale;
  return EP_OK;
}

ep_status ep_net_destroy(ep_net *n) {
  if (!n) return EP_OK;
  UNet &u = n->u;
  if (u.st) cudaStreamSynchronize(u.st);
  for (float *p : u.act) cudaFree(p);
  for (float *p : u.grad) cudaFree(p);
  cudaFree(u.scratch); cudaFree(u.scratch2);
  cudaFree(u.w); cudaFree(u.g); cudaFree(u.m); cudaFree(u.v); cudaFree(u.wb); cudaFree(u.dloss);
  cudaFree(u.wpk); cudaFree(u.xcl); cudaFree(u.terr);
  delete n;
  return EP_OK;
}

const char *ep_net_last_error(ep_net *n) { return n ? n->err.c_str() : g_net_err.c_str(); }

}  // extern "C"
