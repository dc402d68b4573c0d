// Device bodies of the regrouping steps (stable partition by the gate bits,
// tile offsets, merge levels), written for any block size so that the
// standalone kernels of regroup.cu and the persistent batched layer kernel
// run the same code.  Each body processes one tile (or one digit, or one
// merge block) and takes its shared memory from the caller.
//
// Tile layout: a tile of THREADS * ITEMS terms; warp w owns the contiguous
// range [w * 32 * ITEMS, (w + 1) * 32 * ITEMS), lane l holds terms
// w * 32 * ITEMS + 32 j + l, so warp-local ranks follow the input order
// (stability).
#pragma once

#include "internal.h"

namespace sv {

constexpr int RG_TILE = SORT_TILE;  // terms per partition tile (shares the radix sort's scan scratch)
constexpr int MG_TILE = 4096;       // outputs per merge block

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

// ---------------------------------------------------------------- counts
struct PartCountsSmem {
  uint32_t h[16];
};

// Number of terms with each local index r in tile t (cnt[r * tiles + t])
// and in total (added to hist[r]).
template <int THREADS, int ITEMS>
__device__ __forceinline__ void part_counts_tile(const uint64_t* __restrict__ keys, uint64_t n, const GateParams& gp,
                                                 uint64_t tiles, uint32_t* __restrict__ cnt,
                                                 uint32_t* __restrict__ hist, uint64_t t, PartCountsSmem& s) {
  static_assert(THREADS * ITEMS == RG_TILE, "partition tiles hold RG_TILE terms");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = gp.m, D = 1 << m;
  int q[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) q[k] = gp.qpos[k];
  if (tid < 16) s.h[tid] = 0;
  __syncthreads();
  const uint64_t base = t * RG_TILE + (uint64_t)warp * 32 * ITEMS + lane;
  uint64_t k[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint64_t idx = base + i * 32;
    k[i] = idx < n ? keys[idx] : 0ull;
  }
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint64_t idx = base + i * 32;
    uint32_t d = 16u;
    if (idx < n) {
      if (gp.direct)
        d = k[i] == ~0ull ? 16u : (uint32_t)k[i] & ((1u << m) - 1u);
      else
        d = (uint32_t)(gp.rmap >> (4 * gate_index_of(k[i], q, m))) & 15u;
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (d < 16 && lane == __ffs(peers) - 1) atomicAdd(&s.h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  if (tid < D) {
    const uint32_t c = s.h[tid];
    cnt[(uint64_t)tid * tiles + t] = c;
    if (c) atomicAdd(&hist[tid], c);
  }
}

// ---------------------------------------------------------------- offsets
template <int THREADS>
struct TileOffsetsSmem {
  uint32_t wsum[THREADS / 32 > 32 ? THREADS / 32 : 32];
  uint32_t carry;
};

// For digit d: off[d * tiles + t] = base(d) + the counts of digit d in the
// tiles before t, base(d) = the number of keys with a smaller digit (hist).
template <int THREADS>
__device__ __forceinline__ void tile_offsets_digit(const uint32_t* __restrict__ cnt,
                                                   const uint32_t* __restrict__ hist, uint64_t tiles,
                                                   uint32_t* __restrict__ off, int d, TileOffsetsSmem<THREADS>& s) {
  constexpr int WARPS = THREADS / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    uint32_t b = 0;
    for (int e = 0; e < d; ++e) b += hist[e];
    s.carry = b;
  }
  __syncthreads();
  const uint32_t* row = cnt + (uint64_t)d * tiles;
  uint32_t* orow = off + (uint64_t)d * tiles;
  for (uint64_t c0 = 0; c0 < tiles; c0 += THREADS) {
    const uint64_t t = c0 + tid;
    const uint32_t v = t < tiles ? row[t] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s.wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = lane < WARPS ? s.wsum[lane] : 0u;
      uint32_t z = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= o) z += y;
      }
      if (lane < WARPS) s.wsum[lane] = z - w;  // exclusive over warps
    }
    __syncthreads();
    const uint32_t carry = s.carry;
    if (t < tiles) orow[t] = carry + s.wsum[warp] + x - v;
    __syncthreads();
    if (tid == THREADS - 1) s.carry = carry + s.wsum[warp] + x;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- scatter
template <int THREADS>
struct PartScatterSmem {
  uint32_t whist[THREADS / 32][16];
  uint32_t out[16];
  uint64_t seg[5];  // read by all lanes alike (broadcast), kept out of the registers
};

// Stable scatter of tile t's new sort keys into the runs: the tile ranks its
// terms per warp and local index and each thread writes its terms straight
// to their places in the runs (the tile's slice of run r starts at
// off[r * tiles + t]).
template <int THREADS, int ITEMS, bool PAIRS>
__device__ __forceinline__ void part_scatter_tile(const uint64_t* __restrict__ keys, uint64_t n, const GateParams& gp,
                                                  uint64_t tiles, const uint32_t* __restrict__ off,
                                                  uint64_t* __restrict__ sk, uint32_t* __restrict__ sidx, uint64_t t,
                                                  PartScatterSmem<THREADS>& s) {
  static_assert(THREADS * ITEMS == RG_TILE, "partition tiles hold RG_TILE terms");
  constexpr int WARPS = THREADS / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = gp.m, D = 1 << m, vb = gp.vbits;
  const uint32_t dmask = (uint32_t)D - 1u;
  int qpos[4], rem[4];
  gate_positions(gp, qpos, rem);
  if (tid == 0) segment_masks(rem, m, s.seg);
  for (int i = tid; i < WARPS * 16; i += THREADS) (&s.whist[0][0])[i] = 0;
  if (tid < D) s.out[tid] = off[(uint64_t)tid * tiles + t];
  __syncthreads();
  const uint64_t base = t * RG_TILE + (uint64_t)warp * 32 * ITEMS + lane;
  uint64_t k[ITEMS];
  uint32_t d[ITEMS], rank[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint64_t idx = base + i * 32;
    bool valid = idx < n;
    uint64_t sv = 0ull;
    if (valid) {
      sv = gp.direct ? keys[idx] : sort_key_masked(keys[idx], qpos, s.seg, m, gp.rmap);
      valid = !(gp.direct && sv == ~0ull);  // a dropped term (batched form) is left out
    }
    k[i] = vb ? ((sv << vb) | idx) : sv;
    d[i] = valid ? (uint32_t)(sv & dmask) : 16u;
  }
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t peers = __match_any_sync(0xffffffffu, d[i]);
    const int leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if (lane == leader && d[i] < 16) {
      old = s.whist[warp][d[i]];
      s.whist[warp][d[i]] = old + __popc(peers);
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    rank[i] = old + __popc(peers & lt_mask);
    __syncwarp();
  }
  __syncthreads();
  if (warp == 0 && lane < D) {  // per run: offsets of the warps within the tile's slice of the run
    uint32_t c = 0;
    for (int w = 0; w < WARPS; ++w) {
      const uint32_t x = s.whist[w][lane];
      s.whist[w][lane] = c;
      c += x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    if (d[i] < 16) {
      const uint64_t o = (uint64_t)s.out[d[i]] + s.whist[warp][d[i]] + rank[i];
      sk[o] = k[i];
      if (PAIRS) sidx[o] = (uint32_t)(base + i * 32);
    }
  }
}

// ---------------------------------------------------------------- merge
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

// Shared memory of one merge block: both slices at padded positions.
inline size_t merge_smem_bytes(bool pairs) {
  return (sizeof(uint64_t) + (pairs ? sizeof(uint32_t) : 0)) * (size_t)mg_pad(MG_TILE);
}

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

// Where merge block b starts in its pair's first run (one warp).
__device__ __forceinline__ void merge_split_warp(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ hist,
                                                 int D, int level, uint32_t b, uint32_t* __restrict__ splits,
                                                 int lane) {
  uint32_t a0, la, lb, o0, o1;
  if (!merge_block(hist, D, level, b, a0, la, lb, o0, o1)) return;
  const uint64_t* A = kin + a0;
  const uint32_t a = merge_path_warp(A, la, A + la, lb, o0, lane);
  if (lane == 0) splits[b] = a;
}

struct MergeHdr {
  uint32_t a0, la, o0, o1, split[2];
  int live;
};

// Merge block b of a level: stage both slices (dyn: merge_smem_bytes), each
// thread merges ITEMS outputs and writes them back through shared memory.
template <int THREADS, int ITEMS, bool PAIRS>
__device__ __forceinline__ void merge_tile(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                           uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                           const uint32_t* __restrict__ hist, int D, int level,
                                           const uint32_t* __restrict__ splits, uint32_t b, MergeHdr& h,
                                           uint8_t* dyn) {
  static_assert(THREADS * ITEMS == MG_TILE, "merge blocks hold MG_TILE outputs");
  uint64_t* s_k = reinterpret_cast<uint64_t*>(dyn);
  uint32_t* s_v = reinterpret_cast<uint32_t*>(dyn + sizeof(uint64_t) * mg_pad(MG_TILE));
  const int tid = threadIdx.x;
  if (tid == 0) {
    uint32_t a0, la, lb, o0, o1;
    const bool live = merge_block(hist, D, level, b, a0, la, lb, o0, o1);
    if (live) {
      h.a0 = a0;
      h.la = la;
      h.o0 = o0;
      h.o1 = o1;
      h.split[0] = splits[b];
      h.split[1] = o1 == la + lb ? la : splits[b + 1];  // the pair's next tile is the next block
    }
    h.live = live;
  }
  __syncthreads();
  if (!h.live) return;
  const uint32_t a0 = h.a0, la = h.la, o0 = h.o0, o1 = h.o1;
  const uint64_t* A = kin + a0;
  const uint32_t ia = h.split[0], na = h.split[1] - ia;
  const uint32_t ib = o0 - ia, nb = (o1 - h.split[1]) - ib;
  const uint32_t len = na + nb;
  {  // stage both slices: all of a thread's loads in flight together
    uint64_t r[ITEMS];
    uint32_t rv[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t e = (uint32_t)tid + (uint32_t)j * THREADS;
      const uint64_t src = e < na ? (uint64_t)ia + e : (uint64_t)la + ib + (e - na);  // from A
      r[j] = 0;
      rv[j] = 0;
      if (e < len) {
        r[j] = A[src];
        if (PAIRS) rv[j] = vin[a0 + src];
      }
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t e = (uint32_t)tid + (uint32_t)j * THREADS;
      if (e < len) {
        s_k[mg_pad(e)] = r[j];
        if (PAIRS) s_v[mg_pad(e)] = rv[j];
      }
    }
  }
  __syncthreads();
  // this thread's outputs: [diag, diag + ITEMS) of the block's slice.
  // Both slices sit in shared memory at padded positions (one gap per 16
  // elements): neighbouring threads read A or B at strides of about 4 or 8
  // elements, which the padding spreads over distinct banks.
  const uint32_t diag = min((uint32_t)tid * ITEMS, len);
  uint32_t lo = diag > nb ? diag - nb : 0u, hi = diag < na ? diag : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (s_k[mg_pad(mid)] <= s_k[mg_pad(na + diag - 1 - mid)])
      lo = mid + 1;
    else
      hi = mid;
  }
  uint32_t pa = lo, pb = diag - lo;
  uint64_t ok[ITEMS];
  uint32_t ov[ITEMS];
  uint64_t ka = pa < na ? s_k[mg_pad(pa)] : 0ull, kb = pb < nb ? s_k[mg_pad(na + pb)] : 0ull;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
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
  for (int j = 0; j < ITEMS; ++j) {
    const uint32_t p = diag + j;
    if (p < len) {
      s_k[mg_pad(p)] = ok[j];
      if (PAIRS) s_v[mg_pad(p)] = ov[j];
    }
  }
  __syncthreads();
  const uint64_t ob = (uint64_t)a0 + o0;
  for (uint32_t j = tid; j < len; j += THREADS) {
    kout[ob + j] = s_k[mg_pad(j)];
    if (PAIRS) vout[ob + j] = s_v[mg_pad(j)];
  }
}

}  // namespace sv
