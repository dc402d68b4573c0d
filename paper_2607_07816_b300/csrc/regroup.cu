// Regrouping by partition and merge: the grouping step of the gate
// application (Sec. IV-A brings contributions to the same basis state
// together before summing them) for a state that is already in the order of
// the previous gate.
//
// Every gate path leaves the state sorted by the sort key of the gate just
// applied: a fixed arrangement of the qubits outside the gate above the gate
// qubits.  The next gate's sort key keeps the qubits outside its own gate in
// the same relative order and moves its gate qubits to the bottom.  Among
// the terms with equal gate bits r the two keys therefore compare alike, so
// the state, split stably by r, consists of 2^m runs that are each already
// sorted by the new key.  The grouping is then one stable partition by r and
// m levels of pairwise merges, instead of a radix sort over all n key bits:
//
//   * counts: per tile of 4096 terms, the number of terms with each r (and
//     the totals per r);
//   * offsets: for every r and tile, the output position of the tile's first
//     term with that r (the radix sort's scan kernel);
//   * scatter: each term's new sort key (the stored key with the gate bits
//     moved to the bottom: a few shifts; the term's index packed below it, or
//     in a separate index array), written stably to its run;
//   * merge levels: runs 2k and 2k+1 are merged into one; a block takes 4096
//     outputs of a merge, whose start in each input run a first kernel finds
//     by a search over the merge path (one warp per block, 32 probes per
//     step, all searches in flight together); the block stages both slices in
//     shared memory, and each thread merges 8 outputs and writes them back
//     through shared memory.
//
// Equal keys cannot occur (basis states are unique), and on ties the left
// run goes first, so the result equals the stable radix sort of the new
// keys bit for bit.
#include "internal.h"
#include "launch.cuh"
#include "regroup.cuh"

namespace sv {

constexpr int RG_THREADS = 512, RG_ITEMS = 8;
static_assert(RG_THREADS * RG_ITEMS == RG_TILE, "partition tiles share the sort's scan kernel and scratch");
constexpr int MG_THREADS = 512, MG_ITEMS = 8;

// Number of terms with each local index r, per tile (cnt[r * tiles + t])
// and in total (hist[r], zeroed by the launcher).
__global__ void __launch_bounds__(RG_THREADS) k_part_counts(const uint64_t* __restrict__ keys, uint64_t n,
                                                            const GateParams gp, uint64_t tiles,
                                                            uint32_t* __restrict__ cnt, uint32_t* __restrict__ hist) {
  pdl_prologue();
  __shared__ PartCountsSmem s;
  part_counts_tile<RG_THREADS, RG_ITEMS>(keys, n, gp, tiles, cnt, hist, blockIdx.x, s);
}

// Stable scatter of the new sort keys into the runs (measured faster than
// staging the tile in shared memory in run order first).  Four blocks per
// SM (32 registers, a few bytes spilled; no shared staging buffer): more
// tiles in flight than three at 40 registers (measured).
template <bool PAIRS>
__global__ void __launch_bounds__(RG_THREADS, 4) k_part_scatter(const uint64_t* __restrict__ keys, uint64_t n,
                                                             const GateParams gp, uint64_t tiles,
                                                             const uint32_t* __restrict__ off,
                                                             uint64_t* __restrict__ sk, uint32_t* __restrict__ sidx) {
  pdl_prologue();
  __shared__ PartScatterSmem<RG_THREADS> s;
  part_scatter_tile<RG_THREADS, RG_ITEMS, PAIRS>(keys, n, gp, tiles, off, sk, sidx, blockIdx.x, s);
}

// Where every block of a merge level starts in its pair's first run: one warp
// per block, all searches in flight together (the merge blocks then start
// without a search of their own).
__global__ void __launch_bounds__(256) k_merge_splits(const uint64_t* __restrict__ kin,
                                                      const uint32_t* __restrict__ hist, int D, int level,
                                                      uint32_t nblocks, uint32_t* __restrict__ splits) {
  pdl_prologue();
  const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= nblocks) return;
  merge_split_warp(kin, hist, D, level, b, splits, threadIdx.x & 31);
}

// Four blocks per SM (measured faster than three).
template <bool PAIRS>
__global__ void __launch_bounds__(MG_THREADS, 4) k_merge_level(const uint64_t* __restrict__ kin,
                                                            const uint32_t* __restrict__ vin,
                                                            uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                            const uint32_t* __restrict__ hist, int D, int level,
                                                            const uint32_t* __restrict__ splits) {
  pdl_prologue();
  extern __shared__ __align__(16) uint8_t s_dyn[];
  __shared__ MergeHdr h;
  merge_tile<MG_THREADS, MG_ITEMS, PAIRS>(kin, vin, kout, vout, hist, D, level, splits, blockIdx.x, h, s_dyn);
}

static size_t merge_smem(bool pairs) { return merge_smem_bytes(pairs); }

cudaError_t regroup_prepare() {
  static DeviceOnce once;
  return once.run([] {
    const int attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_merge_level<true>, (cudaFuncAttribute)attr, (int)merge_smem(true));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_merge_level<false>, (cudaFuncAttribute)attr, (int)merge_smem(false));
    return e;
  });
}

int regroup_terms(const uint64_t* keys, uint64_t n, const GateParams& gp, uint64_t* sk[2], uint32_t* sidx[2],
                  const SortScratch& sc, cudaStream_t st, int* launches, cudaError_t* cerr) {
  const bool pairs = gp.vbits == 0;
  const int m = gp.m, D = 1 << m;
  const uint64_t tiles = (n + RG_TILE - 1) / RG_TILE;
  *launches = 0;
  *cerr = regroup_prepare();
  if (*cerr != cudaSuccess) return 0;
  if (n == 0) return 0;
  if (tiles > sc.lookback_tiles || n > 0xffffffffull || m < 1 || m > 4) {
    *cerr = cudaErrorInvalidValue;
    return 0;
  }
  uint32_t* cnt = reinterpret_cast<uint32_t*>(sc.lookback);
  uint32_t* off = cnt + (uint64_t)D * tiles;
  // sc.hist[0..15] arrives cleared (the gate's table upload clears it)
  launch_pdl(k_part_counts, (unsigned)tiles, RG_THREADS, 0, st, keys, n, gp, tiles, cnt, sc.hist);
  launch_tile_offsets(cnt, sc.hist, tiles, D, off, st);
  if (pairs)
    launch_pdl(k_part_scatter<true>, (unsigned)tiles, RG_THREADS, 0, st, keys, n, gp, tiles, off,
               sk[0], sidx[0]);
  else
    launch_pdl(k_part_scatter<false>, (unsigned)tiles, RG_THREADS, 0, st, keys, n, gp, tiles, off,
               sk[0], nullptr);
  *launches = 3;
  int cur = 0;
  const uint64_t grid = (n + MG_TILE - 1) / MG_TILE + (uint64_t)D;
  uint32_t* splits = cnt;  // the partition's counts and offsets are no longer needed
  for (int level = 1; level <= m; ++level) {
    launch_pdl(k_merge_splits, (unsigned)((grid * 32 + 255) / 256), 256, 0, st, sk[cur], sc.hist, D, level,
               (uint32_t)grid, splits);
    if (pairs)
      launch_pdl(k_merge_level<true>, (unsigned)grid, MG_THREADS, merge_smem(true), st, sk[cur], sidx[cur],
                 sk[1 - cur], sidx[1 - cur], sc.hist, D, level, splits);
    else
      launch_pdl(k_merge_level<false>, (unsigned)grid, MG_THREADS, merge_smem(false), st, sk[cur], nullptr,
                 sk[1 - cur], nullptr, sc.hist, D, level, splits);
    cur ^= 1;
    *launches += 2;
  }
  *cerr = cudaGetLastError();
  return cur;
}

}  // namespace sv
