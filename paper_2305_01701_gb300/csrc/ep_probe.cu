// ep_probe.cu -- measured arithmetic roofs of the device the library runs on.
//
// The FP64 sweeps are bound by FP64 arithmetic on GB300, not by HBM, so their
// roofline needs the device's FP64 rate: a kernel of independent FP64 fused
// multiply-adds held in registers (no memory traffic), timed with CUDA events.
#include <cuda_runtime.h>

#include <string>

#include "ep_internal.cuh"

namespace ep {
namespace {

constexpr int kChains = 8;  // independent accumulation chains per thread

__global__ void k_fma64(double *sink, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // a store the compiler cannot drop, never taken for the arguments used
  if (s == 12345.678) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace ep

extern "C" ep_status ep_measure_fp64_peak(double *tflops) {
  using namespace ep;
  if (!tflops) return EP_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return EP_ERR_CUDA;
  double *sink = nullptr;
  if (cudaMalloc((void **)&sink, sizeof(double) * 4096) != cudaSuccess) return EP_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int threads = 256, blocks = sms * 8, iters = 4096;
  // a = 1 - 2^-30, b = 2^-31: the chains stay finite and never equal the sink test
  const double a = 1.0 - 1.0 / (1 << 30), b = 1.0 / 2147483648.0;
  k_fma64<<<blocks, threads>>>(sink, 64, a, b);   // warm-up
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    k_fma64<<<blocks, threads>>>(sink, iters, a, b);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) return EP_ERR_CUDA;
  const double flops = 2.0 * kChains * (double)iters * threads * blocks;
  *tflops = flops / (best * 1e-3) / 1e12;
  return EP_OK;
}
