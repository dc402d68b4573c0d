// FP64 pipe throughput probe (sv_probe_fp64 in include/sv.h).
//
// The complex128 mat-vec is bound by the FP64 pipe, so its roofline needs
// that pipe's rate on the GPU at hand.  This probe keeps every SM's FP64
// units busy with independent fused multiply-add chains (8 per thread, no
// loads in the loop) and times them with CUDA events on the default stream.
#include <cuda_runtime.h>

#include "sv.h"

namespace {

constexpr int PROBE_THREADS = 256, PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dfma(uint64_t iters, double seed, double* out) {
  double a[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = seed + (threadIdx.x + c) * 1e-9;
  const double x = 1.0 - 1e-12, y = 1e-13;
  for (uint64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = __fma_rn(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += a[c];
  if (s == 12345.678) out[blockIdx.x] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" sv_status sv_probe_fp64(uint64_t iters, int blocks_per_sm, double* tflops, double* ms) {
  if (!tflops || iters == 0 || blocks_per_sm < 1 || blocks_per_sm > 32) return SV_E_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return SV_E_CUDA;
  }
  const unsigned blocks = (unsigned)(sms * blocks_per_sm);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_probe_dfma<<<blocks, PROBE_THREADS>>>(iters / 8 + 1, 0.5, nullptr);  // warm-up
    e = cudaEventRecord(e0);
  }
  if (e == cudaSuccess) {
    k_probe_dfma<<<blocks, PROBE_THREADS>>>(iters, 0.5, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SV_E_CUDA;
  }
  const double fmas = (double)blocks * PROBE_THREADS * PROBE_CHAINS * (double)iters;
  *tflops = 2.0 * fmas / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return SV_OK;
}
