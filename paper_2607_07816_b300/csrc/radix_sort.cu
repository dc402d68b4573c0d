// Stable LSD radix sort of (uint64 key, uint32 value) pairs, or of keys
// alone (a key may carry its payload in the bits below the sorted ones).
//
// This is the grouping step of the gate application: contributions to the
// same basis state must be brought together before they are summed (the
// segmented sum of Sec. IV-A), and sorting on the bits outside the gate makes
// every partner group contiguous.  It is also used by the canonical readout.
//
// One histogram kernel counts every 8-bit digit in one read.  Each pass then
// runs three kernels with no waiting between blocks: the digit counts of
// every tile, their exclusive scan over the tiles for every digit (plus the
// digit's base from the global histogram), and the scatter, in which a tile
// ranks its keys per warp with __match_any_sync, stages them in shared
// memory in digit order and writes each digit run at its scanned offset.
#include "internal.h"
#include "launch.cuh"
#include "regroup.cuh"

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

// Tile layout shared by the counting and scatter kernels: tile t holds keys
// [t * SORT_TILE, ...); warp w of the tile owns [w*32*ITEMS, (w+1)*32*ITEMS)
// lane-interleaved, so warp-local ranks follow the input order (stability).
constexpr int ST_WARPS = SORT_THREADS / 32;

__device__ __forceinline__ uint32_t sort_digit(uint64_t k, int shift) {
  return (uint32_t)((k >> shift) & (RADIX - 1));
}

// 1. Digit counts of every tile: cnt[d * tiles + t].
__global__ void __launch_bounds__(SORT_THREADS) k_tile_counts(const uint64_t* __restrict__ kin, uint64_t n,
                                                              int shift, uint64_t tiles,
                                                              uint32_t* __restrict__ cnt) {
  __shared__ uint32_t h[RADIX];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < RADIX; i += SORT_THREADS) h[i] = 0;
  __syncthreads();
  const uint64_t t = blockIdx.x;
  const uint64_t base = t * SORT_TILE;
  uint64_t k[SORT_ITEMS];
#pragma unroll
  for (int i = 0; i < SORT_ITEMS; ++i) {
    const uint64_t idx = base + (uint64_t)warp * 32 * SORT_ITEMS + i * 32 + lane;
    k[i] = idx < n ? kin[idx] : 0ull;
  }
#pragma unroll
  for (int i = 0; i < SORT_ITEMS; ++i) {
    const uint64_t idx = base + (uint64_t)warp * 32 * SORT_ITEMS + i * 32 + lane;
    const uint32_t d = idx < n ? sort_digit(k[i], shift) : (uint32_t)RADIX;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (d < RADIX && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int d = tid; d < RADIX; d += SORT_THREADS) cnt[(uint64_t)d * tiles + t] = h[d];
}

// 2. One block per digit: off[d * tiles + t] = base(d) + counts of digit d in
// tiles before t, base(d) = number of keys with a smaller digit (from the
// global histogram of this pass).
constexpr int SCAN_THREADS = 1024;

__global__ void __launch_bounds__(SCAN_THREADS) k_tile_offsets(const uint32_t* __restrict__ cnt,
                                                               const uint32_t* __restrict__ hist, uint64_t tiles,
                                                               uint32_t* __restrict__ off) {
  pdl_prologue();
  __shared__ TileOffsetsSmem<SCAN_THREADS> s;
  tile_offsets_digit<SCAN_THREADS>(cnt, hist, tiles, off, blockIdx.x, s);
}

void launch_tile_offsets(const uint32_t* cnt, const uint32_t* hist, uint64_t tiles, int digits, uint32_t* off,
                         cudaStream_t st) {
  launch_pdl(k_tile_offsets, digits, SCAN_THREADS, 0, st, cnt, hist, tiles, off);
}

// 3. Scatter: rank the tile's keys per warp (match_any and per-warp digit
// counters), turn the counters into per-warp offsets within each digit, scan
// the tile's digit counts, stage the tile in shared memory in digit order
// and write every digit run at off[d * tiles + t].  PAIRS = false sorts the
// keys alone.
template <bool PAIRS>
__global__ void __launch_bounds__(SORT_THREADS) k_tile_scatter(const uint64_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin,
                                                               uint64_t* __restrict__ kout,
                                                               uint32_t* __restrict__ vout, uint64_t n, int shift,
                                                               uint64_t tiles, const uint32_t* __restrict__ off) {
  static_assert(SORT_THREADS >= RADIX, "one thread per digit");
  extern __shared__ __align__(16) uint8_t s_dyn[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(s_dyn);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_dyn + sizeof(uint64_t) * SORT_TILE);
  __shared__ uint32_t s_whist[ST_WARPS][RADIX];
  __shared__ uint32_t s_local[RADIX];
  __shared__ uint32_t s_out[RADIX];
  __shared__ uint32_t s_wtot[ST_WARPS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t t = blockIdx.x;
  const uint64_t base = t * SORT_TILE;
  for (int i = tid; i < ST_WARPS * RADIX; i += SORT_THREADS) (&s_whist[0][0])[i] = 0;
  if (tid < RADIX) s_out[tid] = off[(uint64_t)tid * tiles + t];
  uint64_t k[SORT_ITEMS];
  uint32_t v[SORT_ITEMS], d[SORT_ITEMS], rank[SORT_ITEMS];
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < SORT_ITEMS; ++i) {
    const uint64_t idx = base + (uint64_t)warp * 32 * SORT_ITEMS + i * 32 + lane;
    const bool valid = idx < n;
    k[i] = valid ? kin[idx] : 0ull;
    v[i] = (PAIRS && valid) ? vin[idx] : 0u;
    d[i] = valid ? sort_digit(k[i], shift) : (uint32_t)RADIX;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < SORT_ITEMS; ++i) {
    const uint32_t peers = __match_any_sync(0xffffffffu, d[i]);
    const int leader = __ffs(peers) - 1;
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
  // per digit: offsets of the warps within the digit, and the digit's count
  uint32_t cnt = 0;
  if (tid < RADIX) {
#pragma unroll
    for (int w = 0; w < ST_WARPS; ++w) {
      const uint32_t c = s_whist[w][tid];
      s_whist[w][tid] = cnt;
      cnt += c;
    }
  }
  // exclusive scan of the digit counts over the tile (threads 0..RADIX-1)
  uint32_t x = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_wtot[warp] = x;
  __syncthreads();
  if (tid < RADIX) {
    uint32_t b = 0;
    for (int w = 0; w < warp; ++w) b += s_wtot[w];
    s_local[tid] = b + x - cnt;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < SORT_ITEMS; ++i) {
    if (d[i] < RADIX) {
      const uint32_t pos = s_local[d[i]] + s_whist[warp][d[i]] + rank[i];
      s_keys[pos] = k[i];
      if (PAIRS) s_vals[pos] = v[i];
    }
  }
  __syncthreads();
  const uint32_t tile_n = (uint32_t)(n - base < (uint64_t)SORT_TILE ? n - base : (uint64_t)SORT_TILE);
  for (uint32_t j = tid; j < tile_n; j += SORT_THREADS) {
    const uint64_t key = s_keys[j];
    const uint32_t dd = sort_digit(key, shift);
    const uint64_t out = (uint64_t)s_out[dd] + (j - s_local[dd]);
    kout[out] = key;
    if (PAIRS) vout[out] = s_vals[j];
  }
}

static size_t scatter_smem(bool pairs) { return (sizeof(uint64_t) + (pairs ? sizeof(uint32_t) : 0)) * SORT_TILE; }

// Kernel attributes (dynamic shared memory) set once, outside any stream
// capture.
cudaError_t sort_prepare() {
  static DeviceOnce once;
  return once.run([] {
    cudaError_t e = cudaFuncSetAttribute(k_tile_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)scatter_smem(true));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tile_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)scatter_smem(false));
    return e;
  });
}

// The passes of one sort: digits at lo + 8p for p < ceil(nbits / 8);
// vA/vB == nullptr sorts keys alone.  The per-tile counts and offsets live
// in sc.lookback (2 * RADIX * tiles 32-bit words).
static int sort_passes(uint64_t* kA, uint32_t* vA, uint64_t* kB, uint32_t* vB, uint64_t n, int lo, int nbits,
                       const SortScratch& sc, cudaStream_t st, int* passes_run, cudaError_t* cerr) {
  const int passes = (nbits + RADIX_BITS - 1) / RADIX_BITS;
  const bool pairs = vA != nullptr;
  int cur = 0, run = 0;
  *cerr = sort_prepare();
  if (*cerr != cudaSuccess) {
    *passes_run = 0;
    return 0;
  }
  const uint64_t tiles = sort_tiles(n);
  if (n > 1) {
    if (tiles > sc.lookback_tiles || n > 0xffffffffull) {
      *cerr = cudaErrorInvalidValue;
      *passes_run = 0;
      return 0;
    }
    uint32_t* cnt = reinterpret_cast<uint32_t*>(sc.lookback);
    uint32_t* off = cnt + RADIX * tiles;
    for (int p = 0; p < passes; ++p) {
      if (sc.hist_host) {  // a pass whose digit is the same for every key is the identity
        const uint32_t* hh = sc.hist_host + p * RADIX;
        bool trivial = false;
        for (int dgt = 0; dgt < RADIX; ++dgt)
          if (hh[dgt] == n) trivial = true;
        if (trivial) continue;
      }
      const int shift = lo + RADIX_BITS * p;
      const uint64_t* ki = cur ? kB : kA;
      const uint32_t* vi = cur ? vB : vA;
      uint64_t* ko = cur ? kA : kB;
      uint32_t* vo = cur ? vA : vB;
      k_tile_counts<<<(unsigned)tiles, SORT_THREADS, 0, st>>>(ki, n, shift, tiles, cnt);
      k_tile_offsets<<<RADIX, SCAN_THREADS, 0, st>>>(cnt, sc.hist + p * RADIX, tiles, off);
      if (pairs)
        k_tile_scatter<true><<<(unsigned)tiles, SORT_THREADS, scatter_smem(true), st>>>(ki, vi, ko, vo, n, shift,
                                                                                         tiles, off);
      else
        k_tile_scatter<false><<<(unsigned)tiles, SORT_THREADS, scatter_smem(false), st>>>(ki, nullptr, ko, nullptr,
                                                                                          n, shift, tiles, off);
      cur ^= 1;
      ++run;
    }
  }
  *passes_run = run;
  *cerr = cudaGetLastError();
  return cur;
}

int radix_sort_pairs(uint64_t* kA, uint32_t* vA, uint64_t* kB, uint32_t* vB, uint64_t n, int nbits,
                     const SortScratch& sc, cudaStream_t st, int* passes_run, cudaError_t* cerr) {
  return sort_passes(kA, vA, kB, vB, n, 0, nbits, sc, st, passes_run, cerr);
}

int radix_sort_keys(uint64_t* kA, uint64_t* kB, uint64_t n, int lo, int nbits, const SortScratch& sc,
                    cudaStream_t st, int* passes_run, cudaError_t* cerr) {
  return sort_passes(kA, nullptr, kB, nullptr, n, lo, nbits, sc, st, passes_run, cerr);
}

}  // namespace sv
