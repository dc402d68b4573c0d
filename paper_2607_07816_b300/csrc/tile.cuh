// Order-preserving tile compaction used by the persistent kernels.
//
// A tile of BLOCK*ITEMS elements is laid out warp by warp: warp w owns the
// contiguous range [w*32*ITEMS, (w+1)*32*ITEMS) and in iteration j its lane l
// holds element w*32*ITEMS + j*32 + l, so consecutive lanes read consecutive
// addresses.  Positions come from warp ballots, a scan over the warps and a
// decoupled look-back over tiles, so kept elements keep their input order.
#pragma once

#include "common.cuh"

namespace sv {

template <int BLOCK, int ITEMS>
struct TileLayout {
  static constexpr int TILE = BLOCK * ITEMS;
  static constexpr int WARPS = BLOCK / 32;
  __device__ static __forceinline__ uint64_t index(uint64_t tile_base, int j) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    return tile_base + (uint64_t)warp * 32 * ITEMS + (uint64_t)j * 32 + lane;
  }
};

// Shared state of one compaction: per-warp totals and the tile's global base.
template <int BLOCK>
struct CompactShared {
  uint32_t warp_excl[BLOCK / 32];
  uint32_t tile_total;
  uint64_t tile_base_out;
};

// flags[j] -> positions pos[j] among the tile's kept elements (input order)
// and cs.tile_total; no cross-tile communication.  All threads must call it.
template <int BLOCK, int ITEMS>
__device__ __forceinline__ void tile_local_positions(const bool (&flags)[ITEMS], uint32_t (&pos)[ITEMS],
                                                     CompactShared<BLOCK>& cs) {
  constexpr int WARPS = BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t run = 0;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    uint32_t b = __ballot_sync(0xffffffffu, flags[j]);
    pos[j] = run + __popc(b & lt);
    run += __popc(b);
  }
  if (lane == 0) cs.warp_excl[warp] = run;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < WARPS ? cs.warp_excl[lane] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane < WARPS) cs.warp_excl[lane] = x - v;
    if (lane == 31) cs.tile_total = x;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) pos[j] += cs.warp_excl[warp];
}

// flags[j] -> local positions pos[j] within the tile; after the call
// cs.tile_base_out holds the global output offset of this tile and
// cs.tile_total its number of kept elements.  All threads must call it.
template <int BLOCK, int ITEMS>
__device__ __forceinline__ void tile_compact(const bool (&flags)[ITEMS], uint32_t (&pos)[ITEMS],
                                             CompactShared<BLOCK>& cs, uint64_t* lookback,
                                             uint64_t tile, uint32_t* err) {
  constexpr int WARPS = BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t run = 0;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    uint32_t b = __ballot_sync(0xffffffffu, flags[j]);
    pos[j] = run + __popc(b & lt);
    run += __popc(b);
  }
  if (lane == 0) cs.warp_excl[warp] = run;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < WARPS ? cs.warp_excl[lane] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane < WARPS) cs.warp_excl[lane] = x - v;
    uint32_t total = __shfl_sync(0xffffffffu, x, 31);
    uint64_t base = lookback_exclusive_warp(lookback, tile, total, err);
    if (lane == 0) {
      cs.tile_total = total;
      cs.tile_base_out = base;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) pos[j] += cs.warp_excl[warp];
}

}  // namespace sv
