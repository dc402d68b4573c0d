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

namespace sv {

constexpr int RG_THREADS = 512, RG_ITEMS = 8, RG_TILE = RG_THREADS * RG_ITEMS;
constexpr int RG_WARPS = RG_THREADS / 32;
static_assert(RG_TILE == SORT_TILE, "partition tiles share the sort's scan kernel and scratch");
constexpr int MG_THREADS = 512, MG_ITEMS = 8, MG_TILE = MG_THREADS * MG_ITEMS;

// Local index r of a stored key: the bits at the gate qubits' stored
// positions qpos[t].
__device__ __forceinline__ uint32_t gate_index_of(uint64_t key, const int* qpos, int m) {
  uint32_t r = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (t < m) r |= (uint32_t)((key >> qpos[t]) & 1ull) << t;
  return r;
}

// The gate's sort key of a stored key: the bits at the gate qubits' stored
// positions rem[] (descending) are removed, the rest closes up and moves up
// by m, and the digit of r (r itself, or a monomial gate's output index:
// rmap) takes the bottom.  Written with masks: seg[i] holds the bits between
// the i-th and the (i+1)-th removed position (seg[0] those above all of them,
// seg[m] those below all); a bit of seg[i] has m - i removed positions below
// it, so it moves up by i.
__device__ __forceinline__ void segment_masks(const int* rem, int m, uint64_t* seg) {
#pragma unroll
  for (int i = 0; i <= 4; ++i) {
    seg[i] = 0;
    if (i > m) continue;
    const int hb = i == 0 ? 64 : rem[i - 1];  // bits below hb ...
    const int lb = i == m ? -1 : rem[i];      // ... and above lb
    const uint64_t upper = hb >= 64 ? ~0ull : ((1ull << hb) - 1ull);
    const uint64_t lower = lb + 1 >= 64 ? ~0ull : ((1ull << (lb + 1)) - 1ull);
    seg[i] = upper & ~lower;
  }
}

__device__ __forceinline__ uint64_t sort_key_masked(uint64_t key, const int* qpos, const uint64_t* seg, int m,
                                                    uint64_t rmap) {
  const uint32_t r = (uint32_t)(rmap >> (4 * gate_index_of(key, qpos, m))) & 15u;
  uint64_t x = key & seg[0];
#pragma unroll
  for (int i = 1; i <= 4; ++i)
    if (i <= m) x |= (key & seg[i]) << i;
  return x | r;
}

__device__ __forceinline__ void gate_positions(const GateParams& gp, int* qpos, int* rem) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    qpos[t] = gp.qpos[t];
    rem[t] = t < gp.m ? gp.qpos[t] : -1;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)  // descending
#pragma unroll
    for (int b = a + 1; b < 4; ++b)
      if (rem[b] > rem[a]) {
        const int t = rem[a];
        rem[a] = rem[b];
        rem[b] = t;
      }
}

// Number of terms with each local index r, per tile (cnt[r * tiles + t])
// and in total (hist[r], zeroed by the launcher).
__global__ void __launch_bounds__(RG_THREADS) k_part_counts(const uint64_t* __restrict__ keys, uint64_t n,
                                                            const GateParams gp, uint64_t tiles,
                                                            uint32_t* __restrict__ cnt, uint32_t* __restrict__ hist) {
  pdl_prologue();
  __shared__ uint32_t h[16];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = gp.m, D = 1 << m;
  int q[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) q[t] = gp.qpos[t];
  if (tid < 16) h[tid] = 0;
  __syncthreads();
  const uint64_t t = blockIdx.x;
  const uint64_t base = t * RG_TILE + (uint64_t)warp * 32 * RG_ITEMS + lane;
  uint64_t k[RG_ITEMS];
#pragma unroll
  for (int i = 0; i < RG_ITEMS; ++i) {
    const uint64_t idx = base + i * 32;
    k[i] = idx < n ? keys[idx] : 0ull;
  }
#pragma unroll
  for (int i = 0; i < RG_ITEMS; ++i) {
    const uint64_t idx = base + i * 32;
    uint32_t d = 16u;
    if (idx < n) {
      if (gp.direct)
        d = k[i] == ~0ull ? 16u : (uint32_t)k[i] & ((1u << m) - 1u);
      else
        d = (uint32_t)(gp.rmap >> (4 * gate_index_of(k[i], q, m))) & 15u;
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (d < 16 && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  if (tid < D) {
    const uint32_t c = h[tid];
    cnt[(uint64_t)tid * tiles + t] = c;
    if (c) atomicAdd(&hist[tid], c);
  }
}

// Stable scatter of the new sort keys into the runs: a tile ranks its terms
// per warp and local index and each thread writes its terms straight to
// their places in the runs (the tile's slice of run r starts at
// off[r * tiles + t]; measured faster than staging the tile in shared memory
// in run order first).
// Four blocks per SM (32 registers, a few bytes spilled; no shared staging
// buffer any more): more tiles in flight than three at 40 registers
// (measured).
template <bool PAIRS>
__global__ void __launch_bounds__(RG_THREADS, 4) k_part_scatter(const uint64_t* __restrict__ keys, uint64_t n,
                                                             const GateParams gp, uint64_t tiles,
                                                             const uint32_t* __restrict__ off,
                                                             uint64_t* __restrict__ sk, uint32_t* __restrict__ sidx) {
  pdl_prologue();
  __shared__ uint32_t s_whist[RG_WARPS][16];
  __shared__ uint32_t s_out[16];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = gp.m, D = 1 << m, vb = gp.vbits;
  const uint32_t dmask = (uint32_t)D - 1u;
  int qpos[4], rem[4];
  gate_positions(gp, qpos, rem);
  __shared__ uint64_t s_seg[5];  // read by all lanes alike (broadcast), kept out of the registers
  if (tid == 0) segment_masks(rem, m, s_seg);
  for (int i = tid; i < RG_WARPS * 16; i += RG_THREADS) (&s_whist[0][0])[i] = 0;
  const uint64_t t = blockIdx.x;
  if (tid < D) s_out[tid] = off[(uint64_t)tid * tiles + t];
  __syncthreads();
  const uint64_t base = t * RG_TILE + (uint64_t)warp * 32 * RG_ITEMS + lane;
  uint64_t k[RG_ITEMS];
  uint32_t d[RG_ITEMS], rank[RG_ITEMS];
#pragma unroll
  for (int i = 0; i < RG_ITEMS; ++i) {
    const uint64_t idx = base + i * 32;
    bool valid = idx < n;
    uint64_t s = 0ull;
    if (valid) {
      s = gp.direct ? keys[idx] : sort_key_masked(keys[idx], qpos, s_seg, m, gp.rmap);
      valid = !(gp.direct && s == ~0ull);  // a dropped term (batched form) is left out
    }
    k[i] = vb ? ((s << vb) | idx) : s;
    d[i] = valid ? (uint32_t)(s & dmask) : 16u;
  }
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < RG_ITEMS; ++i) {
    const uint32_t peers = __match_any_sync(0xffffffffu, d[i]);
    const int leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if (lane == leader && d[i] < 16) {
      old = s_whist[warp][d[i]];
      s_whist[warp][d[i]] = old + __popc(peers);
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    rank[i] = old + __popc(peers & lt_mask);
    __syncwarp();
  }
  __syncthreads();
  if (warp == 0 && lane < D) {  // per run: offsets of the warps within the tile's slice of the run
    uint32_t cnt = 0;
    for (int w = 0; w < RG_WARPS; ++w) {
      const uint32_t c = s_whist[w][lane];
      s_whist[w][lane] = cnt;
      cnt += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < RG_ITEMS; ++i) {
    if (d[i] < 16) {
      const uint64_t o = (uint64_t)s_out[d[i]] + s_whist[warp][d[i]] + rank[i];
      sk[o] = k[i];
      if (PAIRS) sidx[o] = (uint32_t)(base + i * 32);
    }
  }
}

// Number of elements of A among the first o outputs of the merge of A and B
// (ties: A first), found by one warp with 32 probes per step.
__device__ __forceinline__ uint32_t merge_path_warp(const uint64_t* __restrict__ A, uint32_t la,
                                                    const uint64_t* __restrict__ B, uint32_t lb, uint32_t o,
                                                    int lane) {
  uint32_t lo = o > lb ? o - lb : 0u, hi = o < la ? o : la;
  while (hi - lo > 32) {
    const uint32_t span = hi - lo;
    const uint32_t x = lo + (uint32_t)(((uint64_t)span * (uint32_t)(lane + 1)) / 33u);
    const bool before = A[x] <= B[o - 1 - x];  // A[x] is among the first o outputs
    const uint32_t bt = __ballot_sync(0xffffffffu, before);
    const int c = __popc(bt);
    const uint32_t x_last = __shfl_sync(0xffffffffu, x, c > 0 ? c - 1 : 0);
    const uint32_t x_first = __shfl_sync(0xffffffffu, x, c < 32 ? c : 31);
    const uint32_t nlo = c > 0 ? x_last + 1 : lo;
    const uint32_t nhi = c < 32 ? x_first : hi;
    lo = nlo;
    hi = nhi;
  }
  const uint32_t x = lo + (uint32_t)lane;
  const bool before = x < hi && A[x] <= B[o - 1 - x];
  return lo + (uint32_t)__popc(__ballot_sync(0xffffffffu, before));
}

__host__ __device__ __forceinline__ constexpr uint32_t mg_pad(uint32_t p) { return p + (p >> 4); }

// One merge level: runs [R(2k L), R((2k+1) L)) and [R((2k+1) L), R((2k+2) L))
// of the input are merged into the same positions of the output, where
// R(e) = hist[0] + ... + hist[e-1] and L = 2^(level-1).  Block b of the
// level takes MG_TILE consecutive outputs of one pair: merge_block finds
// which, and false for blocks past the last pair's last tile.
__device__ __forceinline__ bool merge_block(const uint32_t* __restrict__ hist, int D, int level, uint32_t b,
                                            uint32_t& a0, uint32_t& la, uint32_t& lb, uint32_t& o0,
                                            uint32_t& o1) {
  uint32_t R[17];
  R[0] = 0;
  for (int e = 0; e < D; ++e) R[e + 1] = R[e] + hist[e];
  const int L = 1 << (level - 1);
  for (int e = 0; e + 2 * L <= D; e += 2 * L) {
    const uint32_t r0 = R[e], r1 = R[e + L], r2 = R[e + 2 * L];
    const uint32_t tiles = (r2 - r0 + MG_TILE - 1) / MG_TILE;
    if (b < tiles) {
      a0 = r0;
      la = r1 - r0;
      lb = r2 - r1;
      o0 = b * MG_TILE;
      o1 = min(b * MG_TILE + MG_TILE, r2 - r0);
      return true;
    }
    b -= tiles;
  }
  return false;
}

// Where every block of a merge level starts in its pair's first run: one warp
// per block, all searches in flight together (the merge blocks then start
// without a search of their own).
__global__ void __launch_bounds__(256) k_merge_splits(const uint64_t* __restrict__ kin,
                                                      const uint32_t* __restrict__ hist, int D, int level,
                                                      uint32_t nblocks, uint32_t* __restrict__ splits) {
  pdl_prologue();
  const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= nblocks) return;
  uint32_t a0, la, lb, o0, o1;
  if (!merge_block(hist, D, level, b, a0, la, lb, o0, o1)) return;
  const uint64_t* A = kin + a0;
  const uint32_t a = merge_path_warp(A, la, A + la, lb, o0, lane);
  if (lane == 0) splits[b] = a;
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
  uint64_t* s_k = reinterpret_cast<uint64_t*>(s_dyn);
  uint32_t* s_v = reinterpret_cast<uint32_t*>(s_dyn + sizeof(uint64_t) * mg_pad(MG_TILE));
  __shared__ uint32_t s_a0, s_la, s_o0, s_o1, s_split[2];
  __shared__ int s_live;
  const int tid = threadIdx.x;
  if (tid == 0) {
    uint32_t a0, la, lb, o0, o1;
    const bool live = merge_block(hist, D, level, blockIdx.x, a0, la, lb, o0, o1);
    if (live) {
      s_a0 = a0;
      s_la = la;
      s_o0 = o0;
      s_o1 = o1;
      s_split[0] = splits[blockIdx.x];
      s_split[1] = o1 == la + lb ? la : splits[blockIdx.x + 1];  // the pair's next tile is the next block
    }
    s_live = live;
  }
  __syncthreads();
  if (!s_live) return;
  const uint32_t a0 = s_a0, la = s_la, o0 = s_o0, o1 = s_o1;
  const uint64_t* A = kin + a0;
  const uint64_t* B = A + la;
  const uint32_t ia = s_split[0], na = s_split[1] - ia;
  const uint32_t ib = o0 - ia, nb = (o1 - s_split[1]) - ib;
  const uint32_t len = na + nb;
  {  // stage both slices: all of a thread's loads in flight together
    uint64_t r[MG_ITEMS];
    uint32_t rv[MG_ITEMS];
#pragma unroll
    for (int j = 0; j < MG_ITEMS; ++j) {
      const uint32_t e = (uint32_t)tid + (uint32_t)j * MG_THREADS;
      const uint64_t src = e < na ? (uint64_t)ia + e : (uint64_t)la + ib + (e - na);  // from A
      r[j] = 0;
      rv[j] = 0;
      if (e < len) {
        r[j] = A[src];
        if (PAIRS) rv[j] = vin[a0 + src];
      }
    }
#pragma unroll
    for (int j = 0; j < MG_ITEMS; ++j) {
      const uint32_t e = (uint32_t)tid + (uint32_t)j * MG_THREADS;
      if (e < len) {
        s_k[mg_pad(e)] = r[j];
        if (PAIRS) s_v[mg_pad(e)] = rv[j];
      }
    }
  }
  __syncthreads();
  // this thread's outputs: [diag, diag + MG_ITEMS) of the block's slice.
  // Both slices sit in shared memory at padded positions (one gap per 16
  // elements): neighbouring threads read A or B at strides of about 4 or 8
  // elements, which the padding spreads over distinct banks.
  const uint32_t diag = min((uint32_t)tid * MG_ITEMS, len);
  uint32_t lo = diag > nb ? diag - nb : 0u, hi = diag < na ? diag : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (s_k[mg_pad(mid)] <= s_k[mg_pad(na + diag - 1 - mid)])
      lo = mid + 1;
    else
      hi = mid;
  }
  uint32_t pa = lo, pb = diag - lo;
  uint64_t ok[MG_ITEMS];
  uint32_t ov[MG_ITEMS];
  uint64_t ka = pa < na ? s_k[mg_pad(pa)] : 0ull, kb = pb < nb ? s_k[mg_pad(na + pb)] : 0ull;
#pragma unroll
  for (int j = 0; j < MG_ITEMS; ++j) {
    ok[j] = 0;
    ov[j] = 0;
    if (diag + j < len) {
      const bool take_a = pb >= nb || (pa < na && ka <= kb);
      const uint32_t src = take_a ? pa : na + pb;
      ok[j] = take_a ? ka : kb;
      if (PAIRS) ov[j] = s_v[mg_pad(src)];
      if (take_a) {
        ++pa;
        if (pa < na) ka = s_k[mg_pad(pa)];
      } else {
        ++pb;
        if (pb < nb) kb = s_k[mg_pad(na + pb)];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < MG_ITEMS; ++j) {
    const uint32_t p = diag + j;
    if (p < len) {
      s_k[mg_pad(p)] = ok[j];
      if (PAIRS) s_v[mg_pad(p)] = ov[j];
    }
  }
  __syncthreads();
  const uint64_t ob = (uint64_t)a0 + o0;
  for (uint32_t j = tid; j < len; j += MG_THREADS) {
    kout[ob + j] = s_k[mg_pad(j)];
    if (PAIRS) vout[ob + j] = s_v[mg_pad(j)];
  }
}

static size_t merge_smem(bool pairs) {
  return (sizeof(uint64_t) + (pairs ? sizeof(uint32_t) : 0)) * (size_t)mg_pad(MG_TILE);
}

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
