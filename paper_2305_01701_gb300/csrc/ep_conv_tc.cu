// ep_conv_tc.cu -- the warm-start network's 3^D convolutions as implicit GEMMs
// on the 5th-generation tensor cores (tcgen05), for its forward pass.
//
// One CTA computes a brick of 128 output voxels (8 x 4 x 4 in 3D, 16 x 8 in
// 2D) for all Cout output channels: D[128 x Cout] = sum over taps and input
// channels of A[128 x Cin] B[Cin x Cout], where A is the input brick shifted by
// the tap and B the tap's weights.  Per pipeline stage (one tap, KC input
// channels):
//   * A arrives by TMA (cp.async.bulk.tensor) from a channels-last BF16 copy
//     of the input, one box of 8 channels x the brick per 8 channels; the
//     tensor map's zero fill outside the volume is the convolution's zero
//     padding;
//   * B arrives by a bulk copy (cp.async.bulk) from weights packed per tap in
//     the MMA's operand layout;
//   * one elected thread issues tcgen05.mma (kind::f16, BF16 x BF16, FP32
//     accumulation in tensor memory) K = 16 at a time and frees the stage with
//     tcgen05.commit.
// Operands use the K-major layout without swizzle: 8 x 16-byte core matrices,
// 128 bytes apart along M/N (stride offset) and one 8-channel region apart
// along K (leading offset).  After the last stage the four warps read their
// 32 accumulator rows (tcgen05.ld), add the bias, apply ReLU and store FP32.
// Every wait is bounded; a wait that runs out sets the error word, the block
// waits (bounded) for the copies it issued, frees its tensor memory and ends.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "ep_internal.cuh"

namespace ep {

namespace {

constexpr int TILE_M = 128;   // output voxels per CTA = accumulator rows
constexpr int STAGES = 4;
constexpr int MAX_N = 128;    // largest Cout (accumulator columns)
constexpr int MAX_KC = 64;    // largest input channels per stage
constexpr long long WAIT_LIMIT = 1ll << 31;   // SM cycles, about a second

struct __align__(1024) ConvSmem {
  __nv_bfloat16 a[STAGES][MAX_KC / 8][TILE_M * 8];   // per stage: KC/8 regions of 128 x 8 channels
  __nv_bfloat16 b[STAGES][MAX_KC * MAX_N];           // per stage: KC/8 regions of Cout x 8 channels
  unsigned long long full[STAGES], empty[STAGES], done;
  unsigned tmem_base;
};

__device__ __forceinline__ unsigned su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mb_init(unsigned long long *b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_expect(unsigned long long *b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mb_try(unsigned long long *b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mb_wait(unsigned long long *b, unsigned parity) {
  const long long t0 = clock64();
  while (!mb_try(b, parity))
    if (clock64() - t0 > WAIT_LIMIT) return false;
  return true;
}

__device__ __forceinline__ void tma_box(void *dst, const CUtensorMap *map, int c, int x, int y, int z, int n,
                                        unsigned long long *bar, int D) {
  if (D == 3)
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];\n" ::"r"(su32(dst)),
        "l"(map), "r"(c), "r"(x), "r"(y), "r"(z), "r"(n), "r"(su32(bar))
        : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(su32(dst)),
        "l"(map), "r"(c), "r"(x), "r"(y), "r"(n), "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}

// shared-memory matrix descriptor, K-major without swizzle
__device__ __forceinline__ unsigned long long mdesc(const void *p, unsigned lbo, unsigned sbo) {
  const unsigned long long a = su32(p);
  return ((a & 0x3FFFFull) >> 4) | ((unsigned long long)(lbo >> 4) << 16) |
         ((unsigned long long)(sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = n
__host__ __device__ constexpr unsigned idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(TILE_M >> 4) << 24);
}


struct ConvArgs {
  const __nv_bfloat16 *wpk;   // weights packed per (tap, 16-channel chunk, 8-channel half, co, 8)
  const float *bias;
  float *y;                   // N x Cout x [Z x] Y x X, FP32
  int *err;
  int D, X, Y, Z, cinp, cout, kc, relu, ncol, taps;
};

template <int D>
__global__ void __launch_bounds__(128, 1) k_conv_tc(const __grid_constant__ CUtensorMap map, const ConvArgs A) {
  extern __shared__ unsigned char smem_raw[];
  ConvSmem &S = *reinterpret_cast<ConvSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int BX = D == 3 ? 8 : 16, BY = D == 3 ? 4 : 8, BZ = D == 3 ? 4 : 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nbx = (A.X + BX - 1) / BX, nby = (A.Y + BY - 1) / BY;
  const int bi = blockIdx.x % nbx, bj = (blockIdx.x / nbx) % nby, bk = blockIdx.x / (nbx * nby);
  const int x0 = bi * BX, y0 = bj * BY, z0 = bk * BZ, n = blockIdx.y;
  const int nq = A.cinp / A.kc, nst = A.taps * nq, cout = A.cout;
  __shared__ int fail_s, consumed_s;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mb_init(&S.full[s], 1); mb_init(&S.empty[s], 1); }
    mb_init(&S.done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fail_s = 0;
    consumed_s = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&S.tmem_base)),
                 "r"(A.ncol)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = S.tmem_base;

  if (warp == 0 && lane == 0) {
    // producer: one tap and kc input channels per stage
    int issued = 0;
    for (int it = 0; it < nst; ++it) {
      const int s = it % STAGES;
      const unsigned ph = (unsigned)(it / STAGES) & 1u;
      if (it >= STAGES && !mb_wait(&S.empty[s], ph ^ 1u)) { atomicExch(&fail_s, 1); break; }
      if (*(volatile int *)&fail_s) break;
      const int tap = it / nq, g = it % nq;
      const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = D == 3 ? tap / 9 - 1 : 0;
      mb_expect(&S.full[s], (unsigned)(A.kc * TILE_M * 2 + A.kc * cout * 2));
      for (int j = 0; j < A.kc / 8; ++j)
        tma_box(S.a[s][j], &map, g * A.kc + 8 * j, x0 + dx, y0 + dy, z0 + dz, n, &S.full[s], D);
      const __nv_bfloat16 *src = A.wpk + ((size_t)tap * (A.cinp / 16) + (size_t)g * (A.kc / 16)) * 2 * cout * 8;
      bulk_copy(S.b[s], src, (unsigned)(A.kc * cout * 2), &S.full[s]);
      issued = it + 1;
    }
    // on a failure, wait (bounded) for every stage issued but not consumed
    __syncwarp(1u);
    if (*(volatile int *)&fail_s) {
      for (int it = *(volatile int *)&consumed_s; it < issued; ++it)
        mb_wait(&S.full[it % STAGES], (unsigned)(it / STAGES) & 1u);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const unsigned id = idesc_bf16(cout);
    for (int it = 0; it < nst; ++it) {
      const int s = it % STAGES;
      if (*(volatile int *)&fail_s) break;
      if (!mb_wait(&S.full[s], (unsigned)(it / STAGES) & 1u)) { atomicExch(&fail_s, 1); break; }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      for (int q = 0; q < A.kc / 16; ++q) {
        const unsigned long long ad = mdesc(S.a[s][2 * q], TILE_M * 16, 128);
        const unsigned long long bd = mdesc(S.b[s] + (size_t)2 * q * cout * 8, (unsigned)cout * 16, 128);
        const unsigned acc = (it > 0 || q > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(id), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       su32(&S.empty[s]))
                   : "memory");
      *(volatile int *)&consumed_s = it + 1;
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     su32(&S.done))
                 : "memory");
  }
  __syncwarp();

  // epilogue: warp w reads accumulator rows 32 w .. 32 w + 31
  const bool ok = mb_wait(&S.done, 0u);
  if (!ok) atomicExch(&fail_s, 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const int m = warp * 32 + lane;
  const int vx = x0 + m % BX, vy = y0 + (m / BX) % BY, vz = z0 + m / (BX * BY);
  const bool inside = vx < A.X && vy < A.Y && vz < A.Z && !*(volatile int *)&fail_s;
  const long long nv = (long long)A.X * A.Y * A.Z;
  const long long vox = ((long long)vz * A.Y + vy) * A.X + vx;
  for (int c0 = 0; c0 < cout; c0 += 16) {
    unsigned r[16];
    const unsigned ta = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    if (inside) {
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int co = c0 + e;
        float v = __uint_as_float(r[e]) + A.bias[co];
        if (A.relu && v < 0.f) v = 0.f;
        A.y[((long long)n * cout + co) * nv + vox] = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && fail_s) atomicExch(A.err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(A.ncol) : "memory");
  }
}

// FP32 N x C x V -> BF16 N x V x Cp (channels last, channels >= C zero)
__global__ void k_to_channels_last(const float *x, int N, int C, long long nv, int cp, __nv_bfloat16 *out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)N * nv * cp;
  if (t >= total) return;
  const int c = (int)(t % cp);
  const long long v = (t / cp) % nv, n = t / (cp * nv);
  out[t] = __float2bfloat16_rn(c < C ? x[(n * C + c) * nv + v] : 0.f);
}

// BF16 co x ci x taps -> the operand layout of ConvSmem.b, per tap and
// 16-channel chunk: [half][co][8 channels]; channels >= ci are zero
__global__ void k_pack_weights(const __nv_bfloat16 *w, int cin, int cout, int taps, int cinp,
                               __nv_bfloat16 *out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)taps * cinp * cout;
  if (t >= total) return;
  const int e = (int)(t % 8);
  const int co = (int)((t / 8) % cout);
  const int h = (int)((t / (8 * cout)) % 2);
  const int q = (int)((t / (16LL * cout)) % (cinp / 16));
  const int tap = (int)(t / (16LL * cout * (cinp / 16)));
  const int ci = 16 * q + 8 * h + e;
  out[t] = ci < cin ? w[((long long)co * cin + ci) * taps + tap] : __float2bfloat16_rn(0.f);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

}  // namespace

bool conv_tc_supported(int k, int cout) { return k == 3 && cout >= 16 && cout <= MAX_N && cout % 16 == 0; }

int conv_tc_cinp(int cin) { return (cin + 15) / 16 * 16; }

void conv_tc_to_channels_last(const float *x, int N, int C, long long nv, int cp, __nv_bfloat16 *out,
                              cudaStream_t st) {
  const long long total = (long long)N * nv * cp;
  k_to_channels_last<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(x, N, C, nv, cp, out);
}

void conv_tc_pack_weights(const __nv_bfloat16 *w, int cin, int cout, int taps, __nv_bfloat16 *out, cudaStream_t st) {
  const int cinp = conv_tc_cinp(cin);
  const long long total = (long long)taps * cinp * cout;
  k_pack_weights<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(w, cin, cout, taps, cinp, out);
}

cudaError_t conv_tc_forward(int D, const __nv_bfloat16 *xcl, int N, int X, int Y, int Z, int cin,
                            const __nv_bfloat16 *wpk, const float *bias, int cout, int relu, float *y, int *err,
                            cudaStream_t st) {
  static bool configured[2] = {false, false};
  // 1 KB for the alignment, and 24 KB of slack behind the operand buffers so
  // that every operand address the descriptors can form stays inside the
  // block's shared memory
  const size_t smem = sizeof(ConvSmem) + 1024 + 24 * 1024;
  if (!configured[D - 2]) {
    cudaError_t e = D == 3 ? cudaFuncSetAttribute(k_conv_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                           : cudaFuncSetAttribute(k_conv_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured[D - 2] = true;
  }
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const int cinp = conv_tc_cinp(cin);
  CUtensorMap map;
  CUresult r;
  if (D == 3) {
    cuuint64_t dims[5] = {(cuuint64_t)cinp, (cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)Z, (cuuint64_t)N};
    cuuint64_t strides[4] = {(cuuint64_t)cinp * 2, (cuuint64_t)cinp * 2 * X, (cuuint64_t)cinp * 2 * X * Y,
                             (cuuint64_t)cinp * 2 * X * Y * Z};
    cuuint32_t box[5] = {8, 8, 4, 4, 1}, es[5] = {1, 1, 1, 1, 1};
    r = fn(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(xcl), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    cuuint64_t dims[4] = {(cuuint64_t)cinp, (cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)N};
    cuuint64_t strides[3] = {(cuuint64_t)cinp * 2, (cuuint64_t)cinp * 2 * X, (cuuint64_t)cinp * 2 * X * Y};
    cuuint32_t box[4] = {8, 16, 8, 1}, es[4] = {1, 1, 1, 1};
    r = fn(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(xcl), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  ConvArgs A;
  A.wpk = wpk; A.bias = bias; A.y = y; A.err = err;
  A.D = D; A.X = X; A.Y = Y; A.Z = D == 3 ? Z : 1; A.cinp = cinp; A.cout = cout; A.relu = relu;
  A.kc = cinp % 64 == 0 ? 64 : (cinp % 32 == 0 ? 32 : 16);
  A.ncol = cout <= 32 ? 32 : (cout <= 64 ? 64 : 128);
  A.taps = D == 3 ? 27 : 9;
  const int BX = D == 3 ? 8 : 16, BY = D == 3 ? 4 : 8, BZ = D == 3 ? 4 : 1;
  const unsigned bricks = (unsigned)(((X + BX - 1) / BX) * ((Y + BY - 1) / BY) * ((A.Z + BZ - 1) / BZ));
  dim3 grid(bricks, (unsigned)N);
  if (D == 3) k_conv_tc<3><<<grid, 128, smem, st>>>(map, A);
  else k_conv_tc<2><<<grid, 128, smem, st>>>(map, A);
  return cudaGetLastError();
}

}  // namespace ep
