// Stable LSD radix sort of (uint64 key, uint32 value) pairs.
//
// This is the grouping step of the gate application: contributions to the
// same basis state must be brought together before they are summed (the
// segmented sum of Sec. IV-A), and sorting on the bits outside the gate makes
// every partner group contiguous.  It is also used by the canonical readout.
//
// One histogram kernel counts every 8-bit digit in one read; each pass is a
// single "onesweep" kernel: a tile ranks its keys per warp with
// __match_any_sync, gets the exclusive digit offsets of all earlier tiles by
// decoupled look-back (bounded waits), stages the tile in shared memory in
// digit order and writes each digit run contiguously.
#include "internal.h"

namespace sv {

__global__ void __launch_bounds__(256) k_digit_hist(const uint64_t* __restrict__ k, uint64_t n,
                                                    int passes, uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[MAX_PASSES][RADIX];
  for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t key = k[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&sh[p][(key >> (RADIX_BITS * p)) & (RADIX - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) {
    uint32_t c = (&sh[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
}

void launch_digit_hist(const uint64_t* k, uint64_t n, int nbits, uint32_t* hist, cudaStream_t st) {
  int passes = (nbits + RADIX_BITS - 1) / RADIX_BITS;
  cudaMemsetAsync(hist, 0, sizeof(uint32_t) * MAX_PASSES * RADIX, st);
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_digit_hist<<<(unsigned)blocks, 256, 0, st>>>(k, n, passes, hist);
}

// Exclusive scan of one value per thread over the block (values of threads
// that have none are 0); all BLOCK threads call it.
template <int BLOCK>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  uint32_t base = 0;
  for (int w = 0; w < warp; ++w) base += warp_tot[w];
  __syncthreads();
  return base + x - v;
}

// One pass of the LSD sort over the 8-bit digit at `shift`.  Warp w of the
// tile owns elements [w*32*ITEMS, (w+1)*32*ITEMS) (lane-interleaved), so the
// warp-local ranks (match_any + a per-warp counter per digit) follow the
// input order and the sort is stable.  Threads 0..255 then own one digit
// each: exclusive offsets across warps, the tile-local digit offsets, and
// the decoupled look-back over earlier tiles for the digit's global base.
// PAIRS = false sorts keys alone (a key may carry its payload in the bits
// below `shift`).
template <int BLOCK, int ITEMS, bool PAIRS>
__global__ void __launch_bounds__(BLOCK) k_onesweep(const uint64_t* __restrict__ kin,
                                                   const uint32_t* __restrict__ vin,
                                                   uint64_t* __restrict__ kout,
                                                   uint32_t* __restrict__ vout, uint64_t n,
                                                   int shift, const uint32_t* __restrict__ hist,
                                                   uint64_t* lookback, uint64_t* tile_counter,
                                                   uint32_t* err) {
  static_assert(BLOCK >= RADIX, "one thread per digit");
  constexpr int TILE = BLOCK * ITEMS;
  constexpr int WARPS = BLOCK / 32;
  extern __shared__ __align__(16) uint8_t s_dyn[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(s_dyn);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_dyn + sizeof(uint64_t) * TILE);
  __shared__ uint32_t s_whist[WARPS][RADIX];
  __shared__ uint32_t s_local[RADIX];
  __shared__ uint64_t s_global[RADIX];
  __shared__ uint32_t s_wtot[WARPS];
  __shared__ uint64_t s_tile;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool digit_thread = tid < RADIX;
  if (tid == 0) s_tile = atomicAdd((unsigned long long*)tile_counter, 1ull);
  for (int i = tid; i < WARPS * RADIX; i += BLOCK) (&s_whist[0][0])[i] = 0;
  const uint32_t digit_base = block_exclusive_scan<BLOCK>(digit_thread ? hist[tid] : 0u, s_wtot);
  const uint64_t tile = s_tile;
  const uint64_t base = tile * TILE;

  uint64_t k[ITEMS];
  uint32_t v[ITEMS], d[ITEMS], rank[ITEMS];
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    uint64_t idx = base + (uint64_t)warp * 32 * ITEMS + i * 32 + lane;
    bool valid = idx < n;
    k[i] = valid ? kin[idx] : 0ull;
    v[i] = (PAIRS && valid) ? vin[idx] : 0u;
    d[i] = valid ? (uint32_t)((k[i] >> shift) & (RADIX - 1)) : (uint32_t)RADIX;
  }
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    uint32_t peers = __match_any_sync(0xffffffffu, d[i]);
    int leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if (lane == leader && d[i] < RADIX) {
      old = s_whist[warp][d[i]];
      s_whist[warp][d[i]] = old + __popc(peers);
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    rank[i] = old + __popc(peers & lt_mask);
    __syncwarp();
  }
  __syncthreads();
  uint32_t cnt = 0;
  if (digit_thread) {
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
      uint32_t c = s_whist[w][tid];
      s_whist[w][tid] = cnt;
      cnt += c;
    }
  }
  const uint32_t local = block_exclusive_scan<BLOCK>(cnt, s_wtot);
  if (digit_thread) {
    s_local[tid] = local;
    uint64_t excl = lookback_exclusive_x4(lookback + tid, RADIX, tile, cnt, err);
    s_global[tid] = digit_base + excl;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    if (d[i] < RADIX) {
      uint32_t pos = s_local[d[i]] + s_whist[warp][d[i]] + rank[i];
      s_keys[pos] = k[i];
      if (PAIRS) s_vals[pos] = v[i];
    }
  }
  __syncthreads();
  uint64_t tile_n = n - base < (uint64_t)TILE ? n - base : (uint64_t)TILE;
  for (uint32_t j = tid; j < tile_n; j += BLOCK) {
    uint64_t key = s_keys[j];
    uint32_t dd = (uint32_t)((key >> shift) & (RADIX - 1));
    uint64_t out = s_global[dd] + (j - s_local[dd]);
    kout[out] = key;
    if (PAIRS) vout[out] = s_vals[j];
  }
}

static size_t onesweep_smem(bool pairs) { return (sizeof(uint64_t) + (pairs ? sizeof(uint32_t) : 0)) * SORT_TILE; }

// Kernel attributes (dynamic shared memory) set once, outside any stream
// capture.
void sort_prepare() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_onesweep<SORT_THREADS, SORT_ITEMS, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)onesweep_smem(true));
    cudaFuncSetAttribute(k_onesweep<SORT_THREADS, SORT_ITEMS, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)onesweep_smem(false));
    attr_set = true;
  }
}

int radix_sort_pairs(uint64_t* kA, uint32_t* vA, uint64_t* kB, uint32_t* vB, uint64_t n, int nbits,
                     const SortScratch& sc, cudaStream_t st, int* passes_run, cudaError_t* cerr) {
  int passes = (nbits + RADIX_BITS - 1) / RADIX_BITS;
  int cur = 0, run = 0;
  *cerr = cudaSuccess;
  sort_prepare();
  uint64_t tiles = sort_tiles(n);
  if (n > 1) {
    for (int p = 0; p < passes; ++p) {
      // a pass whose digit is the same for every key is the identity (known
      // only when the caller read the histograms back: hist_host != NULL)
      if (sc.hist_host) {
        const uint32_t* hh = sc.hist_host + p * RADIX;
        bool trivial = false;
        for (int dgt = 0; dgt < RADIX; ++dgt)
          if (hh[dgt] == n) trivial = true;
        if (trivial) continue;
      }
      if (tiles > sc.lookback_tiles) {
        *cerr = cudaErrorInvalidValue;
        return cur;
      }
      cudaMemsetAsync(sc.lookback, 0, sizeof(uint64_t) * RADIX * tiles, st);
      cudaMemsetAsync(sc.tile_counter, 0, sizeof(uint64_t), st);
      const uint64_t* ki = cur ? kB : kA;
      const uint32_t* vi = cur ? vB : vA;
      uint64_t* ko = cur ? kA : kB;
      uint32_t* vo = cur ? vA : vB;
      k_onesweep<SORT_THREADS, SORT_ITEMS, true><<<(unsigned)tiles, SORT_THREADS, onesweep_smem(true), st>>>(
          ki, vi, ko, vo, n, RADIX_BITS * p, sc.hist + p * RADIX, sc.lookback, sc.tile_counter,
          sc.err);
      cur ^= 1;
      ++run;
    }
  }
  *passes_run = run;
  *cerr = cudaGetLastError();
  return cur;
}

int radix_sort_keys(uint64_t* kA, uint64_t* kB, uint64_t n, int lo, int nbits, const SortScratch& sc,
                    cudaStream_t st, int* passes_run, cudaError_t* cerr) {
  const int passes = (nbits + RADIX_BITS - 1) / RADIX_BITS;
  int cur = 0, run = 0;
  *cerr = cudaSuccess;
  sort_prepare();
  const uint64_t tiles = sort_tiles(n);
  if (n > 1) {
    for (int p = 0; p < passes; ++p) {
      if (sc.hist_host) {  // a pass whose digit is the same for every key is the identity
        const uint32_t* hh = sc.hist_host + p * RADIX;
        bool trivial = false;
        for (int dgt = 0; dgt < RADIX; ++dgt)
          if (hh[dgt] == n) trivial = true;
        if (trivial) continue;
      }
      if (tiles > sc.lookback_tiles) {
        *cerr = cudaErrorInvalidValue;
        return cur;
      }
      cudaMemsetAsync(sc.lookback, 0, sizeof(uint64_t) * RADIX * tiles, st);
      cudaMemsetAsync(sc.tile_counter, 0, sizeof(uint64_t), st);
      const uint64_t* ki = cur ? kB : kA;
      uint64_t* ko = cur ? kA : kB;
      k_onesweep<SORT_THREADS, SORT_ITEMS, false><<<(unsigned)tiles, SORT_THREADS, onesweep_smem(false), st>>>(
          ki, nullptr, ko, nullptr, n, lo + RADIX_BITS * p, sc.hist + p * RADIX, sc.lookback, sc.tile_counter,
          sc.err);
      cur ^= 1;
      ++run;
    }
  }
  *passes_run = run;
  *cerr = cudaGetLastError();
  return cur;
}

}  // namespace sv
