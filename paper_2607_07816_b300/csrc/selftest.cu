// Device self-tests of the conversion-free complex64 helpers against the
// conversion instructions they stand in for (sv_selftest in include/sv.h).
#include <cuda_runtime.h>

#include "c64_exact.cuh"
#include "common.cuh"
#include "sv.h"

namespace sv {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x) {  // splitmix64 finaliser
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// A float drawn to cover the cases that matter: random bit patterns over the
// whole finite range, subnormals, few-bit significands (exact ties), and
// magnitudes near a given exponent.
__device__ float draw_float(uint64_t h, int near_exp) {
  const uint32_t kind = (uint32_t)(h >> 60);
  const uint32_t r = (uint32_t)h;
  const uint32_t sign = (uint32_t)(h >> 59) << 31;
  uint32_t bits;
  if (kind < 4) {  // any finite float
    bits = r & 0x7fffffffu;
    if ((bits >> 23) == 0xff) bits &= 0x7f7fffffu;
  } else if (kind < 6) {  // subnormal
    bits = r & 0x7fffffu;
  } else if (kind < 10) {  // few significand bits
    const uint32_t e = 1u + ((r >> 8) % 253u);
    bits = (e << 23) | ((r & 0xffu) << 15);
  } else {  // near 2^near_exp, random significand
    int e = near_exp + (int)((r >> 24) % 7u) - 3 + 127;
    e = e < 1 ? 1 : (e > 254 ? 254 : e);
    bits = ((uint32_t)e << 23) | (r & 0x7fffffu);
  }
  return __uint_as_float(sign | bits);
}

__device__ double draw_scale(uint64_t h) {
  const uint32_t kind = (uint32_t)(h >> 61);
  uint64_t m = h & ((1ull << 52) - 1);
  if (kind < 3) m &= 0xFFull << 44;  // few bits: products with ties
  const int e = (int)((h >> 52) % 48u) - 8;  // 2^-8 .. 2^39
  return __longlong_as_double((long long)(((uint64_t)(e + 1023) << 52) | m));
}

__global__ void k_selftest(int which, uint64_t n, uint64_t seed, unsigned long long* bad,
                           unsigned long long* first) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t h1 = mix64(seed ^ (2 * i)), h2 = mix64(seed ^ (2 * i + 1));
    bool ok;
    if (which == 0) {
      const float re = draw_float(h1, 0);
      // im: anywhere, or about 26 binades below re (its square then sits at
      // the rounding position of re^2: ties and near-ties)
      const int ere = (int)((__float_as_uint(re) >> 23) & 0xffu) - 127;
      const float im = draw_float(h2, ((h2 >> 58) & 1u) ? ere - 26 - (int)((h2 >> 40) & 3u) : ere);
      const double want = __fma_rn((double)re, (double)re, __dmul_rn((double)im, (double)im));
      ok = amp_prob_bits(re, im) == (uint64_t)__double_as_longlong(want);
    } else {
      const float x = draw_float(h1, -(int)((h1 >> 32) % 140u));
      const double s = draw_scale(h2);
      const float want = __double2float_rn(__dmul_rn((double)x, s));
      ok = __float_as_uint(scaled_f32_mul(x, s)) == __float_as_uint(want);
    }
    if (!ok) {
      atomicAdd(bad, 1ull);
      atomicMin(first, (unsigned long long)i);
    }
  }
}

// A bounded wait that runs out: tile 1 waits for tile 0's descriptor, which
// nothing publishes.  The kernel must give up after the poll limit, flag
// ERR_TIMEOUT and return normally.
__global__ void k_wait_runs_out(uint64_t* lb, uint32_t* err, uint32_t limit) {
  lookback_exclusive_warp(lb, 1, 5, err, limit);
}

}  // namespace
}  // namespace sv

static sv_status selftest_wait(uint64_t* mismatches, uint64_t* first_bad) {
  uint64_t* lb = nullptr;
  uint32_t* err = nullptr;
  if (cudaMalloc(&lb, 4 * sizeof(uint64_t)) != cudaSuccess || cudaMalloc(&err, sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(lb);
    return SV_E_NOMEM;
  }
  cudaError_t e = cudaMemset(lb, 0, 4 * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(uint32_t));
  if (e == cudaSuccess) {
    sv::k_wait_runs_out<<<1, 32>>>(lb, err, 1u << 14);
    e = cudaGetLastError();
  }
  uint32_t flags = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flags, err, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  cudaFree(lb);
  cudaFree(err);
  if (e != cudaSuccess) return SV_E_CUDA;
  *mismatches = (flags & sv::ERR_TIMEOUT) ? 0 : 1;
  *first_bad = flags;
  return SV_OK;
}

extern "C" sv_status sv_selftest(int which, uint64_t n, uint64_t seed, uint64_t* mismatches, uint64_t* first_bad) {
  if ((which < 0 || which > 2) || !mismatches || !first_bad) return SV_E_ARG;
  if (which == 2) return selftest_wait(mismatches, first_bad);
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return SV_E_NOMEM;
  }
  const unsigned long long init[2] = {0ull, ~0ull};
  cudaError_t e = cudaMemcpy(d, init, sizeof(init), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n > 0) {
    sv::k_selftest<<<148 * 4, 256>>>(which, n, seed, d, d + 1);
    e = cudaGetLastError();
  }
  unsigned long long out[2] = {0ull, ~0ull};
  if (e == cudaSuccess) e = cudaMemcpy(out, d, sizeof(out), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return SV_E_CUDA;
  *mismatches = out[0];
  *first_bad = out[1];
  return SV_OK;
}
