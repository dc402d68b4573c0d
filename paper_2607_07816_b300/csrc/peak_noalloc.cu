// sv_peak_noalloc: the most probable term of a caller-owned, device-resident
// term list, computed without allocating any memory.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// want the readout -- code whose device memory belongs to another runtime
// or memory pool that forbids outside allocations, processes running under
// a fixed device-memory budget, and code paths where an allocation would
// synchronise the device at a bad time.  They pass their own key and
// amplitude arrays and get the peak back; the only working memory used is a
// fixed array compiled into this library.
//
// The scratch is one file-scope device array (NA_SCRATCH_BYTES, 64 KiB +
// 256 B).  Every GPU that loads the library holds it until the process
// exits.  It holds one partial result per block, so a call handles at most
// NA_MAX_TERMS = 4096 blocks x 65536 terms = 2^28 terms; larger inputs are
// rejected with SV_E_ARG.  All calls on a device share the array and it
// keeps the last call's contents: the block ticket is cleared at the start
// of every call, and calls that overlap on the GPU (two streams, or two host
// threads) race on it.
#include <atomic>
#include <cstring>

#include "internal.h"
#include "sv.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr uint64_t NA_CHUNK = 1ull << 16;   // terms reduced by one block
constexpr int NA_MAX_BLOCKS = 4096;
constexpr uint64_t NA_MAX_TERMS = NA_CHUNK * NA_MAX_BLOCKS;
// layout: partial prob bits [4096] | partial keys [4096] | ticket | result (prob bits, key)
constexpr size_t NA_OFF_KEYS = sizeof(uint64_t) * NA_MAX_BLOCKS;
constexpr size_t NA_OFF_TICKET = 2 * sizeof(uint64_t) * NA_MAX_BLOCKS;
constexpr size_t NA_OFF_RESULT = NA_OFF_TICKET + 64;
constexpr size_t NA_SCRATCH_BYTES = NA_OFF_RESULT + 192;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

// Device address of g_noalloc_scratch, looked up once per device.
constexpr int NA_MAX_DEVICES = 64;
std::atomic<void*> g_scratch_addr[NA_MAX_DEVICES];

__device__ __forceinline__ bool better(uint64_t p1, uint64_t k1, uint64_t p2, uint64_t k2) {
  return p1 > p2 || (p1 == p2 && k1 < k2);
}

__device__ __forceinline__ void block_best(uint64_t& bp, uint64_t& bk) {
  __shared__ uint64_t sp[NA_THREADS / 32], sk[NA_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t p = __shfl_down_sync(0xffffffffu, (unsigned long long)bp, o);
    uint64_t k = __shfl_down_sync(0xffffffffu, (unsigned long long)bk, o);
    if (better(p, k, bp, bk)) {
      bp = p;
      bk = k;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sp[warp] = bp;
    sk[warp] = bk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NA_THREADS / 32; ++w)
      if (better(sp[w], sk[w], bp, bk)) {
        bp = sp[w];
        bk = sk[w];
      }
  }
}

template <typename C2>
__global__ void __launch_bounds__(NA_THREADS) k_peak_noalloc(const uint64_t* __restrict__ keys,
                                                            const C2* __restrict__ amps, uint64_t n,
                                                            unsigned char* scratch) {
  uint64_t* part_p = reinterpret_cast<uint64_t*>(scratch);
  uint64_t* part_k = reinterpret_cast<uint64_t*>(scratch + NA_OFF_KEYS);
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + NA_OFF_TICKET);
  uint64_t* result = reinterpret_cast<uint64_t*>(scratch + NA_OFF_RESULT);
  __shared__ bool s_last;
  const uint64_t begin = blockIdx.x * NA_CHUNK;
  const uint64_t end = begin + NA_CHUNK < n ? begin + NA_CHUNK : n;
  uint64_t bp = 0, bk = ~0ull;
  for (uint64_t i = begin + threadIdx.x; i < end; i += NA_THREADS) {
    C2 a = amps[i];
    uint64_t p = (uint64_t)__double_as_longlong(sv::prob_of((double)a.x, (double)a.y));
    uint64_t k = keys[i];
    if (better(p, k, bp, bk)) {
      bp = p;
      bk = k;
    }
  }
  block_best(bp, bk);
  if (threadIdx.x == 0) {
    part_p[blockIdx.x] = bp;
    part_k[blockIdx.x] = bk;
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  // last block: reduce the per-block partials
  __threadfence();
  bp = 0;
  bk = ~0ull;
  for (uint32_t b = threadIdx.x; b < gridDim.x; b += NA_THREADS) {
    uint64_t p = ((volatile uint64_t*)part_p)[b], k = ((volatile uint64_t*)part_k)[b];
    if (better(p, k, bp, bk)) {
      bp = p;
      bk = k;
    }
  }
  block_best(bp, bk);
  if (threadIdx.x == 0) {
    result[0] = bp;
    result[1] = bk;
  }
}

}  // namespace

extern "C" sv_status sv_peak_noalloc(int prec, const uint64_t* keys, const void* amps, uint64_t n,
                                     void* cuda_stream, uint64_t* key, double* prob) {
  if ((prec != SV_C128 && prec != SV_C64) || !keys || !amps || !key || !prob) return SV_E_ARG;
  if (n == 0 || n > NA_MAX_TERMS) return SV_E_ARG;  // empty, or beyond the fixed scratch (2^28 terms)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    cudaGetLastError();
    return SV_E_CUDA;
  }
  // one-time set-up on this device: the device address of the scratch
  void* base = g_scratch_addr[dev].load();
  if (!base) {
    if (cudaGetSymbolAddress(&base, g_noalloc_scratch) != cudaSuccess || !base) {
      cudaGetLastError();
      return SV_E_CUDA;
    }
    g_scratch_addr[dev].store(base);
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned char* scratch = static_cast<unsigned char*>(base);
  if (cudaMemsetAsync(scratch + NA_OFF_TICKET, 0, sizeof(unsigned int), st) != cudaSuccess) {
    cudaGetLastError();
    return SV_E_CUDA;
  }
  const unsigned blocks = (unsigned)((n + NA_CHUNK - 1) / NA_CHUNK);
  if (prec == SV_C128)
    k_peak_noalloc<double2><<<blocks, NA_THREADS, 0, st>>>(keys, (const double2*)amps, n, scratch);
  else
    k_peak_noalloc<float2><<<blocks, NA_THREADS, 0, st>>>(keys, (const float2*)amps, n, scratch);
  uint64_t out[2] = {0, 0};
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, scratch + NA_OFF_RESULT, sizeof(out), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SV_E_CUDA;
  }
  *key = out[1];
  double p;
  static_assert(sizeof(p) == sizeof(out[0]), "bit copy");
  memcpy(&p, &out[0], sizeof(p));
  *prob = p;
  return SV_OK;
}
