// Batched form: many independent circuits in one segmented state.
//
// Every term carries the id of the circuit (segment) it belongs to, and the
// segments are contiguous in the buffers.  One step applies one gate to each
// segment (Eq. 3, Sec. IV-A, with each segment's own qubits and unitary) and
// then truncates each segment to its own top-k (Sec. III): the whole batch
// goes through one key transform, one grouping sort (segment id in the top
// bits of the sort key, so groups never mix segments and the output stays
// grouped by segment), one mat-vec pass, one segmented radix select and one
// renormalising compaction, instead of the same pipeline once per circuit.
// The arithmetic per group and the cut per segment are those of the single
// state path, so each segment's result is the one it would get alone.
#include "internal.h"
#include "launch.cuh"
#include "tile.cuh"
#include "batch.h"
#include "c64_exact.cuh"
#include "select.cuh"
#include "regroup.cuh"

namespace sv {

// ---------------------------------------------------------------- keys
// The nibble tables of each slot's sort order for this step (one block per
// slot): fwd[k][v] = the sort-key bits of natural bits 4k.. given by v,
// inv[k][v] = the natural bits of sort-key bits 4k.. given by v.
struct SegTablesSmem {
  int8_t nat[64];  // sort-key bit -> qubit
};

// The tables of one slot; blockDim.x == 256 (one thread per table word).
__device__ __forceinline__ void seg_tables_slot(const SegGate* __restrict__ gates, uint64_t* __restrict__ tables,
                                                uint32_t slot, SegTablesSmem& s) {
  const SegGate& gt = gates[slot];
  uint64_t* fwd = tables + (uint64_t)slot * SEG_TABLE_WORDS;
  uint64_t* inv = fwd + 256;
  if (threadIdx.x < 64) s.nat[threadIdx.x] = -1;
  __syncthreads();
  if (gt.m < 0) return;  // removed or free slot: no tables needed
  if (threadIdx.x < 64) {
    const int p = gt.pos[threadIdx.x];
    if (p < 64) s.nat[p] = (int8_t)threadIdx.x;
  }
  __syncthreads();
  const int k = threadIdx.x >> 4, v = threadIdx.x & 15;
  uint64_t f = 0, g = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if ((v >> j) & 1) {
      const int b = 4 * k + j;
      if (gt.pos[b] < 64) f |= 1ull << gt.pos[b];
      if (s.nat[b] >= 0) g |= 1ull << s.nat[b];
    }
  fwd[threadIdx.x] = f;
  inv[threadIdx.x] = g;
}

__global__ void __launch_bounds__(256) k_seg_tables(const SegGate* __restrict__ gates,
                                                    uint64_t* __restrict__ tables) {
  __shared__ SegTablesSmem s;
  seg_tables_slot(gates, tables, blockIdx.x, s);
}

void launch_seg_tables(const SegGate* gates, int slots, uint64_t* tables, cudaStream_t st) {
  if (slots > 0) k_seg_tables<<<slots, 256, 0, st>>>(gates, tables);
}

__device__ __forceinline__ uint64_t nibble_map(const uint64_t* __restrict__ t, uint64_t x) {
  uint64_t y = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) y |= t[16 * k + ((x >> (4 * k)) & 15u)];
  return y;
}

// Sort key of every term: (segment rank, the key in its slot's sort order),
// all ones for a term of a removed segment (left out of the grouping).
__device__ __forceinline__ void seg_keys_range(const uint64_t* __restrict__ keys, const uint16_t* __restrict__ seg,
                                               uint64_t n, const SegGate* __restrict__ gates,
                                               const uint64_t* __restrict__ tables, int shift,
                                               uint64_t* __restrict__ sk, uint64_t first, uint64_t stride) {
  for (uint64_t i = first; i < n; i += stride) {
    const uint32_t sg = seg[i];
    uint64_t s = ~0ull;
    if (gates[sg].m >= 0)
      s = ((uint64_t)gates[sg].rank << shift) | nibble_map(tables + (uint64_t)sg * SEG_TABLE_WORDS, keys[i]);
    sk[i] = s;
  }
}

__global__ void __launch_bounds__(256) k_seg_keys(const uint64_t* __restrict__ keys,
                                                  const uint16_t* __restrict__ seg, uint64_t n,
                                                  const SegGate* __restrict__ gates,
                                                  const uint64_t* __restrict__ tables, int shift,
                                                  uint64_t* __restrict__ sk) {
  seg_keys_range(keys, seg, n, gates, tables, shift, sk, blockIdx.x * (uint64_t)blockDim.x + threadIdx.x,
                 (uint64_t)gridDim.x * blockDim.x);
}

void launch_seg_keys(const uint64_t* keys, const uint16_t* seg, uint64_t n, const SegGate* gates,
                     const uint64_t* tables, int shift, uint64_t* sk, cudaStream_t st) {
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_seg_keys<<<(unsigned)blocks, 256, 0, st>>>(keys, seg, n, gates, tables, shift, sk);
}

// ---------------------------------------------------------------- heads
constexpr int SH_BLOCK = 256, SH_ITEMS = 16;

__device__ __forceinline__ uint64_t seg_group_key(uint64_t s, int shift, const SegGate* gates,
                                                  const uint16_t* rank_slot) {
  const uint32_t sg = rank_slot[(uint32_t)(s >> shift)];
  return s >> gates[sg].m;  // the segment rank stays in the top bits
}

struct SegHeadsSmem {
  CompactShared<SH_BLOCK> cs;
  uint64_t tile;
};

// Group heads of the grouped sort keys, tiles taken from
// ctl->tile_counter[0] until none is left; the group count lands in
// ctl->count[0].
__device__ __forceinline__ void seg_heads_run(const uint64_t* __restrict__ sk, uint64_t n, int shift,
                                              const SegGate* __restrict__ gates,
                                              const uint16_t* __restrict__ rank_slot, uint32_t* __restrict__ heads,
                                              uint64_t* lookback, Ctl* ctl, SegHeadsSmem& s) {
  typedef TileLayout<SH_BLOCK, SH_ITEMS> L;
  const uint64_t tiles = (n + L::TILE - 1) / L::TILE;
  while (true) {
    if (threadIdx.x == 0) s.tile = atomicAdd((unsigned long long*)&ctl->tile_counter[0], 1ull);
    __syncthreads();
    const uint64_t tile = s.tile;
    if (tile >= tiles) break;
    const uint64_t base = tile * L::TILE;
    bool flag[SH_ITEMS];
    uint32_t pos[SH_ITEMS];
#pragma unroll
    for (int j = 0; j < SH_ITEMS; ++j) {
      const uint64_t i = L::index(base, j);
      bool f = false;
      if (i < n) {
        const uint64_t a = sk[i];
        f = i == 0 || (a >> shift) != (sk[i - 1] >> shift) ||
            seg_group_key(a, shift, gates, rank_slot) != seg_group_key(sk[i - 1], shift, gates, rank_slot);
      }
      flag[j] = f;
    }
    tile_compact<SH_BLOCK, SH_ITEMS>(flag, pos, s.cs, lookback, tile, &ctl->err);
#pragma unroll
    for (int j = 0; j < SH_ITEMS; ++j)
      if (flag[j]) heads[s.cs.tile_base_out + pos[j]] = (uint32_t)L::index(base, j);
    if (tile == tiles - 1 && threadIdx.x == 0) ctl->count[0] = s.cs.tile_base_out + s.cs.tile_total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SH_BLOCK) k_seg_heads(const uint64_t* __restrict__ sk, uint64_t n, int shift,
                                                        const SegGate* __restrict__ gates,
                                                        const uint16_t* __restrict__ rank_slot,
                                                        uint32_t* __restrict__ heads, uint64_t* lookback,
                                                        Ctl* ctl) {
  __shared__ SegHeadsSmem s;
  seg_heads_run(sk, n, shift, gates, rank_slot, heads, lookback, ctl, s);
}

void launch_seg_heads(const uint64_t* sk, uint64_t n, int shift, const SegGate* gates, const uint16_t* rank_slot,
                      uint32_t* heads,
                      uint64_t* lookback, Ctl* ctl, cudaStream_t st) {
  const uint64_t tiles = (n + SH_BLOCK * SH_ITEMS - 1) / (SH_BLOCK * SH_ITEMS);
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * (tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[0], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[0], 0, sizeof(uint64_t), st);
  if (n == 0) return;
  const uint64_t grid = tiles < 148 * 4 ? tiles : 148 * 4;
  k_seg_heads<<<(unsigned)grid, SH_BLOCK, 0, st>>>(sk, n, shift, gates, rank_slot, heads, lookback, ctl);
}

// ---------------------------------------------------------------- segment bounds
// Where each slot's terms start and end in an output list, recorded while
// the list is written: output i of a tile of `total` outputs written from
// position base, whose slots are sl[0..total).  Slot changes inside the tile
// are marked at once; the tile's first and last outputs may continue a slot
// from the neighbouring tiles, so their marks take the minimum (start) and
// maximum (end).  start must arrive all ones and end zero; a slot with no
// outputs keeps them.
__device__ __forceinline__ void seg_bound_marks(const uint16_t* sl, uint32_t i, uint32_t total, uint64_t base,
                                                uint64_t* __restrict__ start, uint64_t* __restrict__ end) {
  if (!start) return;
  const uint16_t s = sl[i];
  if (i == 0 || sl[i - 1] != s) atomicMin((unsigned long long*)&start[s], (unsigned long long)(base + i));
  if (i + 1 == total || sl[i + 1] != s) atomicMax((unsigned long long*)&end[s], (unsigned long long)(base + i + 1));
}

// ---------------------------------------------------------------- apply
template <typename Real>
struct SCplx;
template <>
struct SCplx<double> {
  typedef double2 T;
};
template <>
struct SCplx<float> {
  typedef float2 T;
};
__device__ __forceinline__ double sfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float sfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

constexpr int SA_BLOCK = 256;

// One thread per partner group (GPT consecutive groups per thread, MAXD =
// 2^mmax outputs per group at most).  A thread reads its group's members
// once, in ascending r, and runs every output's fused multiply-add chain in
// registers (the single-state order, U rounded to the amplitude precision,
// products with a zero U component skipped).  Nonzero outputs are placed in
// (group, r') order: a block scan of the per-thread counts and a decoupled
// look-back over tiles give each thread its output range.  With hist1 the
// write-back also counts every output in its slot's histogram of the
// select's first digit (the select's first level then needs no scan).
struct SegApplySmem {
  uint32_t warp[SA_BLOCK / 32];
  uint64_t base;
  uint32_t total;
  uint64_t tile;
  uint32_t hslot;   // slot whose first-digit counts hcnt holds (~0: none)
  uint32_t* hcnt;   // [SEL_BINS] in shared memory
};

// Add the block's first-digit counts of slot sm.hslot to the slot's global
// histogram and clear them (all threads call it).
__device__ __forceinline__ void seg_hist1_flush(SegApplySmem& sm, uint32_t* __restrict__ hist1) {
  const uint32_t sl = sm.hslot;
  if (sl != 0xffffffffu)
    for (int b = threadIdx.x; b < SEL_BINS; b += SA_BLOCK) {
      const uint32_t c = sm.hcnt[b];
      if (c) {
        atomicAdd(&hist1[(uint64_t)sl * SEL_BINS + b], c);
        sm.hcnt[b] = 0;
      }
    }
}

template <typename Real, int MAXD, int GPT>
__device__ __forceinline__ void seg_apply_run(
    const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sidx, uint64_t n,
    const uint32_t* __restrict__ heads, const typename SCplx<Real>::T* __restrict__ amps_in, int shift,
    const SegGate* __restrict__ gates, const uint16_t* __restrict__ rank_slot, const uint64_t* __restrict__ keys_in,
    uint64_t* __restrict__ keys_out,
    typename SCplx<Real>::T* __restrict__ amps_out, uint64_t* __restrict__ probs_out,
    uint16_t* __restrict__ seg_out, uint32_t* __restrict__ hist1, uint64_t* __restrict__ start,
    uint64_t* __restrict__ end, uint64_t* lookback, uint64_t max_tiles, Ctl* ctl, SegApplySmem& sm, uint8_t* s_dyn) {
  typedef typename SCplx<Real>::T C2;
  constexpr int TILE_G = SA_BLOCK * GPT;
  constexpr int WARPS = SA_BLOCK / 32;
  constexpr int NOUT = SA_BLOCK * GPT * MAXD;  // most outputs of one tile
  // a tile's outputs are staged in shared memory and written back coalesced
  // (a thread's outputs are consecutive, so direct stores of neighbouring
  // threads fall 2^m apart)
  uint64_t* s_ok = reinterpret_cast<uint64_t*>(s_dyn);
  uint64_t* s_op = s_ok + NOUT;
  C2* s_oa = reinterpret_cast<C2*>(s_op + NOUT);
  uint16_t* s_os = reinterpret_cast<uint16_t*>(s_oa + NOUT);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t G = ctl->count[0];
  const uint64_t tiles = (G + TILE_G - 1) / TILE_G;
  if (tiles > max_tiles) {  // the look-back buffer was sized for fewer tiles
    if (tid == 0) atomicOr(&ctl->err, ERR_INVARIANT);
    return;
  }
  if (hist1) {
    for (int b = tid; b < SEL_BINS; b += SA_BLOCK) sm.hcnt[b] = 0;
    if (tid == 0) sm.hslot = 0xffffffffu;
  }
  while (true) {
    if (tid == 0) sm.tile = atomicAdd((unsigned long long*)&ctl->tile_counter[1], 1ull);
    __syncthreads();
    const uint64_t tile = sm.tile;
    if (tile >= tiles) break;
    const uint64_t g0 = tile * TILE_G + (uint64_t)tid * GPT;
    Real yr[GPT][MAXD], yi[GPT][MAXD];
    uint32_t keep[GPT], qpack[GPT];
    int mj[GPT];
    uint64_t rest[GPT];
    uint16_t sgj[GPT];
    uint32_t cnt = 0;
    // the loads of the GPT groups are issued together, level by level
    // (heads, first sort key and index, first amplitude): most groups of a
    // truncated state have a single member
    uint64_t hb[GPT + 1], s0v[GPT], k0v[GPT];
    C2 x0v[GPT];
#pragma unroll
    for (int j = 0; j <= GPT; ++j) {
      const uint64_t g = g0 + j;
      hb[j] = g < G ? (uint64_t)heads[g] : n;
    }
#pragma unroll
    for (int j = 0; j < GPT; ++j) {
      const bool ok = g0 + j < G;
      s0v[j] = ok ? sk[hb[j]] : 0ull;
      const uint32_t ix = ok ? sidx[hb[j]] : 0u;
      x0v[j] = ok ? amps_in[ix] : C2();
      k0v[j] = ok ? keys_in[ix] : 0ull;  // the head member's natural key
    }
#pragma unroll
    for (int j = 0; j < GPT; ++j) {
      keep[j] = 0;
      qpack[j] = 0;
      mj[j] = 0;
      rest[j] = 0;
      sgj[j] = 0;
#pragma unroll
      for (int ro = 0; ro < MAXD; ++ro) yr[j][ro] = yi[j][ro] = (Real)0;
      const uint64_t g = g0 + j;
      if (g >= G) continue;
      const uint64_t h = hb[j];
      const uint64_t e = hb[j + 1];
      const uint64_t s0 = s0v[j];
      const uint32_t sg = rank_slot[(uint32_t)(s0 >> shift)];
      const SegGate& gt = gates[sg];
      const int m = gt.m;
      const int d = 1 << m;
      for (uint64_t i = h; i < e; ++i) {
        const uint32_t r = (uint32_t)((i == h ? s0 : sk[i]) & (uint64_t)(d - 1));
        const C2 x = i == h ? x0v[j] : amps_in[sidx[i]];
#pragma unroll
        for (int ro = 0; ro < MAXD; ++ro) {
          if (ro >= d) break;
          const bool rnz = (gt.re_nz[ro] >> r) & 1u, inz = (gt.im_nz[ro] >> r) & 1u;
          if (rnz) {
            const Real ur = (Real)gt.U[2 * (ro * d + r)];
            yr[j][ro] = sfma(ur, x.x, yr[j][ro]);
            yi[j][ro] = sfma(ur, x.y, yi[j][ro]);
          }
          if (inz) {
            const Real ui = (Real)gt.U[2 * (ro * d + r) + 1];
            yr[j][ro] = sfma(-ui, x.y, yr[j][ro]);
            yi[j][ro] = sfma(ui, x.x, yi[j][ro]);
          }
        }
      }
#pragma unroll
      for (int ro = 0; ro < MAXD; ++ro)
        if (ro < d && !(yr[j][ro] == (Real)0 && yi[j][ro] == (Real)0)) keep[j] |= 1u << ro;
      uint64_t qmask = 0;
      for (int t = 0; t < m; ++t) {
        qpack[j] |= (uint32_t)gt.q[t] << (8 * t);
        qmask |= 1ull << gt.q[t];
      }
      mj[j] = m;
      // the group's natural key without the gate bits: any member's natural
      // key (the batched state keeps natural keys) with the gate bits cleared
      rest[j] = k0v[j] & ~qmask;
      sgj[j] = (uint16_t)sg;
      cnt += __popc(keep[j]);
    }
    // block exclusive scan of the counts, then the tile's global base
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sm.warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const uint32_t v = lane < WARPS ? sm.warp[lane] : 0u;
      uint32_t w = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < WARPS) sm.warp[lane] = w - v;
      const uint32_t total = __shfl_sync(0xffffffffu, w, 31);
      const uint64_t base = lookback_exclusive_warp(lookback, tile, total, &ctl->err);
      if (lane == 0) {
        sm.total = total;
        sm.base = base;
      }
    }
    __syncthreads();
    uint32_t o = sm.warp[warp] + (x - cnt);  // position within the tile's outputs
#pragma unroll
    for (int j = 0; j < GPT; ++j) {
      if (!keep[j]) continue;
      int q[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) q[t] = (int)((qpack[j] >> (8 * t)) & 0xffu);
#pragma unroll
      for (int ro = 0; ro < MAXD; ++ro) {
        if (!((keep[j] >> ro) & 1u)) continue;
        s_ok[o] = rest[j] | seg_deposit_r((uint32_t)ro, q, mj[j]);
        C2 y;
        y.x = yr[j][ro];
        y.y = yi[j][ro];
        s_oa[o] = y;
        s_op[o] = amp_prob_bits(yr[j][ro], yi[j][ro]);
        s_os[o] = sgj[j];
        ++o;
      }
    }
    __syncthreads();
    const uint64_t base = sm.base;
    if (hist1 && sm.total > 0 && s_os[0] != sm.hslot) {
      // the block's counts follow the slot of its tiles' first outputs: a
      // change of slot flushes them (tiles come in increasing order)
      seg_hist1_flush(sm, hist1);
      __syncthreads();
      if (tid == 0) sm.hslot = s_os[0];
      __syncthreads();
    }
    for (uint32_t i0 = 0; i0 < sm.total; i0 += SA_BLOCK) {
      const uint32_t i = i0 + (uint32_t)tid;
      uint32_t hk = 0xffffffffu;
      if (i < sm.total) {
        keys_out[base + i] = s_ok[i];
        amps_out[base + i] = s_oa[i];
        probs_out[base + i] = s_op[i];
        seg_out[base + i] = s_os[i];
        hk = ((uint32_t)s_os[i] << SEL_BITS) | sel_first_digit(s_op[i]);
        seg_bound_marks(s_os, i, sm.total, base, start, end);
      }
      if (hist1) {  // the select's first digit per slot (lanes of one slot and digit add once)
        const uint32_t peers = __match_any_sync(0xffffffffu, hk);
        if (hk != 0xffffffffu && lane == __ffs(peers) - 1) {
          const uint32_t sl = hk >> SEL_BITS, dg = hk & (SEL_BINS - 1);
          if (sl == sm.hslot)
            atomicAdd(&sm.hcnt[dg], (uint32_t)__popc(peers));
          else  // a tile that reaches into the next slot
            atomicAdd(&hist1[(uint64_t)sl * SEL_BINS + dg], (uint32_t)__popc(peers));
        }
      }
    }
    if (tile == tiles - 1 && tid == 0) ctl->count[1] = sm.base + sm.total;
    __syncthreads();
  }
  if (hist1) seg_hist1_flush(sm, hist1);
}

template <typename Real, int MAXD, int GPT>
__global__ void __launch_bounds__(SA_BLOCK) k_seg_apply(
    const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sidx, uint64_t n,
    const uint32_t* __restrict__ heads, const typename SCplx<Real>::T* __restrict__ amps_in, int shift,
    const SegGate* __restrict__ gates, const uint16_t* __restrict__ rank_slot, const uint64_t* __restrict__ keys_in,
    uint64_t* __restrict__ keys_out,
    typename SCplx<Real>::T* __restrict__ amps_out, uint64_t* __restrict__ probs_out,
    uint16_t* __restrict__ seg_out, uint32_t* __restrict__ hist1, uint64_t* __restrict__ start,
    uint64_t* __restrict__ end, uint64_t* lookback, uint64_t max_tiles, Ctl* ctl) {
  extern __shared__ __align__(16) uint8_t s_dyn[];
  __shared__ SegApplySmem sm;
  __shared__ uint32_t s_hcnt[SEL_BINS];
  if (threadIdx.x == 0) sm.hcnt = s_hcnt;
  __syncthreads();
  seg_apply_run<Real, MAXD, GPT>(sk, sidx, n, heads, amps_in, shift, gates, rank_slot, keys_in, keys_out, amps_out,
                                 probs_out, seg_out, hist1, start, end, lookback, max_tiles, ctl, sm, s_dyn);
}

// Shared staging of one tile's outputs: key, probability, amplitude, slot.
template <typename C2>
__host__ __device__ constexpr size_t seg_apply_smem(int maxd, int gpt) {
  return (size_t)SA_BLOCK * gpt * maxd * (8 + 8 + sizeof(C2) + 2);
}

template <typename Real, int MAXD, int GPT>
cudaError_t seg_apply_attr() {
  typedef typename SCplx<Real>::T C2;
  return cudaFuncSetAttribute(k_seg_apply<Real, MAXD, GPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)seg_apply_smem<C2>(MAXD, GPT));
}

template <typename Real>
cudaError_t seg_apply_attrs() {
  cudaError_t e = seg_apply_attr<Real, 2, 1>();
  if (e == cudaSuccess) e = seg_apply_attr<Real, 2, 2>();
  if (e == cudaSuccess) e = seg_apply_attr<Real, 2, 4>();
  if (e == cudaSuccess) e = seg_apply_attr<Real, 4, 1>();
  if (e == cudaSuccess) e = seg_apply_attr<Real, 4, 2>();
  if (e == cudaSuccess) e = seg_apply_attr<Real, 4, 4>();
  if (e == cudaSuccess) e = seg_apply_attr<Real, 8, 1>();
  if (e == cudaSuccess) e = seg_apply_attr<Real, 8, 2>();
  if (e == cudaSuccess) e = seg_apply_attr<Real, 16, 1>();
  return e;
}

template <typename Real>
void seg_apply_dispatch(int mmax, int gpt, unsigned grid, cudaStream_t st, const uint64_t* sk, const uint32_t* sidx,
                        uint64_t n, const uint32_t* heads, const void* amps_in, int shift, const SegGate* gates,
                        const uint16_t* rank_slot, const uint64_t* keys_in, uint64_t* keys_out, void* amps_out,
                        uint64_t* probs_out,
                        uint16_t* seg_out, uint32_t* hist1, uint64_t* start, uint64_t* end,
                        uint64_t* lookback, uint64_t max_tiles, Ctl* ctl) {
  typedef typename SCplx<Real>::T C2;
  const C2* ai = (const C2*)amps_in;
  C2* ao = (C2*)amps_out;
#define SV_SEG_APPLY(MAXD, GPT)                                                                         \
  k_seg_apply<Real, MAXD, GPT><<<grid, SA_BLOCK, seg_apply_smem<C2>(MAXD, GPT), st>>>(                    \
      sk, sidx, n, heads, ai, shift, gates, rank_slot, keys_in, keys_out, ao, probs_out, seg_out, hist1, start, \
      end, lookback, max_tiles, ctl)
  if (mmax <= 1) {
    if (gpt == 1) SV_SEG_APPLY(2, 1);
    else if (gpt == 2) SV_SEG_APPLY(2, 2);
    else SV_SEG_APPLY(2, 4);
  } else if (mmax == 2) {
    if (gpt == 1) SV_SEG_APPLY(4, 1);
    else if (gpt == 2) SV_SEG_APPLY(4, 2);
    else SV_SEG_APPLY(4, 4);
  } else if (mmax == 3) {
    if (gpt == 1) SV_SEG_APPLY(8, 1);
    else SV_SEG_APPLY(8, 2);
  } else {
    SV_SEG_APPLY(16, 1);
  }
#undef SV_SEG_APPLY
}

int seg_apply_configs(int mmax) { return mmax <= 2 ? 3 : (mmax == 3 ? 2 : 1); }

// cfg picks the groups per thread (1, 2 or 4 where the accumulators fit);
// max_tiles bounds the look-back buffer: at least groups / 256 + 1, the tile
// count of one group per thread.
void launch_seg_apply(int prec, const uint64_t* sk, const uint32_t* sidx, uint64_t n, const uint32_t* heads,
                      const void* amps_in, int shift, int mmax, const SegGate* gates, const uint16_t* rank_slot,
                      const uint64_t* keys_in, uint64_t* keys_out, void* amps_out, uint64_t* probs_out,
                      uint16_t* seg_out, uint32_t* hist1, uint64_t* start, uint64_t* end,
                      uint64_t* lookback, Ctl* ctl, uint64_t max_tiles, int cfg, cudaStream_t st) {
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * (max_tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[1], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[1], 0, sizeof(uint64_t), st);
  if (n == 0) return;
  const int ncfg = seg_apply_configs(mmax);
  const int gpt = 1 << (cfg < ncfg ? cfg : ncfg - 1);
  const uint64_t grid = max_tiles < 148 * 4 ? (max_tiles ? max_tiles : 1) : 148 * 4;
  if (prec == 0)
    seg_apply_dispatch<double>(mmax, gpt, (unsigned)grid, st, sk, sidx, n, heads, amps_in, shift, gates, rank_slot,
                               keys_in, keys_out, amps_out, probs_out, seg_out, hist1, start, end, lookback, max_tiles,
                               ctl);
  else
    seg_apply_dispatch<float>(mmax, gpt, (unsigned)grid, st, sk, sidx, n, heads, amps_in, shift, gates, rank_slot,
                              keys_in, keys_out, amps_out, probs_out, seg_out, hist1, start, end, lookback, max_tiles,
                              ctl);
}

// ---------------------------------------------------------------- segmented select
// The single-state radix select run for every segment at once, top-k only:
// each segment has its own select state (prefix of the select key
// z = (~prob_bits, key), target rank, count before its bin).  A level scans
// all terms in contiguous chunks, walked as runs of one segment each.  While
// a segment's bin is large the scan builds its digit histogram (counts only:
// the rank decides the bin); once the bin holds at most SF_CAP terms, the
// next scan copies them out for the finish kernel and sums, in the exact
// fixed point of the masses, the segment's total mass and the mass of the
// terms ranked before the bin.  The cut's mass is then the latter plus the
// masses of the bin's terms up to the cut, added by the finish kernel.
constexpr int SS_BINS = SEL_BINS;
constexpr int SS_BLOCK = 256, SS_ILP = 4;
constexpr int SF_CAP = SEGSEL_CAP;

// A segment whose current bin holds at most SF_CAP terms is in collect mode.
__device__ __forceinline__ bool seg_collects(const SegSel& st) {
  return st.active && !st.done && st.bin_count <= (uint64_t)SF_CAP;
}

// Is z ranked before (strictly above) every key under the bits-long prefix?
__device__ __forceinline__ bool z_before_prefix(uint64_t hi, uint64_t lo, uint64_t ph, uint64_t pl, int bits) {
  if (bits <= 64) return (hi >> (64 - bits)) < (ph >> (64 - bits));
  if (hi != ph) return hi < ph;
  return (lo >> (128 - bits)) < (pl >> (128 - bits));
}


struct SegHistSmem {
  uint32_t cnt[SS_BINS];
  u128 part[2][SS_BLOCK / 32];
  uint32_t seg;
};

// One level's scan by block `cta` of `ncta`: a contiguous chunk of the terms.
__device__ __forceinline__ void segsel_hist_chunk(const uint64_t* __restrict__ probs,
                                                          const uint64_t* __restrict__ keys,
                                                          const uint16_t* __restrict__ seg,
                                                          const uint64_t* __restrict__ n_dev,
                                                          const SegSel* __restrict__ sel,
                                                          uint32_t* __restrict__ g_cnt, uint64_t* __restrict__ g_sum,
                                                          uint64_t* __restrict__ g_buf, uint32_t* __restrict__ g_bufn,
                                                          uint32_t* err, uint32_t cta, uint32_t ncta,
                                                          SegHistSmem& sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // one contiguous chunk per block, whole multiples of a block's sweep
  const uint64_t n = *n_dev;
  const uint64_t sweep = (uint64_t)SS_BLOCK * SS_ILP;
  uint64_t chunk = (n + ncta - 1) / ncta;
  chunk = (chunk + sweep - 1) / sweep * sweep;
  if (chunk < 4 * sweep) chunk = 4 * sweep;
  const uint64_t c0 = cta * chunk;
  if (c0 >= n) return;
  const uint64_t c1 = c0 + chunk < n ? c0 + chunk : n;
  uint64_t i0 = c0;
  while (i0 < c1) {
    if (tid == 0) sm.seg = seg[i0];
    __syncthreads();
    const uint32_t sg = sm.seg;
    const SegSel& st = sel[sg];
    const bool collect = seg_collects(st);
    const bool count = st.active && !st.done && !collect;
    const int bits = (int)st.bits;
    const uint64_t ph = st.prefix_hi, pl = st.prefix_lo;
    int D, sh;
    sel_digit(bits, &D, &sh);
    uint64_t i1;
    {  // end of the run: first index in [i0, c1) of another segment
      uint64_t lo = i0, hi = c1;
      while (lo < hi) {
        const uint64_t mid = (lo + hi) / 2;
        if (seg[mid] == sg) lo = mid + 1;
        else hi = mid;
      }
      i1 = lo;
    }
    if (count) {
      for (int b = tid; b < SS_BINS; b += SS_BLOCK) sm.cnt[b] = 0;
      __syncthreads();
      const bool need_lo = bits > 64 || sh < 64;
      for (uint64_t b0 = i0; b0 < i1; b0 += (uint64_t)SS_BLOCK * SS_ILP) {
        uint64_t pb[SS_ILP];
#pragma unroll
        for (int u = 0; u < SS_ILP; ++u) {
          const uint64_t i = b0 + (uint64_t)u * SS_BLOCK + tid;
          pb[u] = i < i1 ? probs[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < SS_ILP; ++u) {
          const uint64_t i = b0 + (uint64_t)u * SS_BLOCK + tid;
          const uint64_t hi = ~pb[u];
          bool act = i < i1 && (bits > 64 || ((hi ^ ph) >> (64 - bits)) == 0);
          const uint64_t lo = act && need_lo ? keys[i] : 0ull;
          if (act && bits > 64) act = z_matches(hi, lo, ph, pl, bits);
          if (bits == 1) {
            // first level: the digit is the exponent, shared by most lanes
            const uint32_t dg = act ? z_digit(hi, lo, sh, D) : 0xffffffffu;
            const uint32_t peers = __match_any_sync(0xffffffffu, dg);
            if (act && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&sm.cnt[dg], (uint32_t)__popc(peers));
          } else if (act) {
            atomicAdd(&sm.cnt[z_digit(hi, lo, sh, D)], 1u);
          }
        }
      }
      __syncthreads();
      uint32_t* gc = g_cnt + (uint64_t)sg * SS_BINS;
      for (int b = tid; b < (1 << D); b += SS_BLOCK)
        if (sm.cnt[b]) atomicAdd(&gc[b], sm.cnt[b]);
    } else if (collect) {
      uint64_t* buf = g_buf + (uint64_t)sg * 2 * SF_CAP;
      u128 tot = 0, above = 0;
      for (uint64_t b0 = i0; b0 < i1; b0 += (uint64_t)SS_BLOCK * SS_ILP) {
        uint64_t pb[SS_ILP];
#pragma unroll
        for (int u = 0; u < SS_ILP; ++u) {
          const uint64_t i = b0 + (uint64_t)u * SS_BLOCK + tid;
          pb[u] = i < i1 ? probs[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < SS_ILP; ++u) {
          const uint64_t i = b0 + (uint64_t)u * SS_BLOCK + tid;
          if (i >= i1) continue;
          const uint64_t hi = ~pb[u];
          const u128 v = fx_from_bits(pb[u], err);
          tot += v;
          if (bits <= 64 && ((hi ^ ph) >> (64 - bits)) != 0) {
            if (z_before_prefix(hi, 0, ph, pl, bits)) above += v;
            continue;
          }
          const uint64_t lo = keys[i];
          if (!z_matches(hi, lo, ph, pl, bits)) {
            if (z_before_prefix(hi, lo, ph, pl, bits)) above += v;
            continue;
          }
          const uint32_t p = atomicAdd(&g_bufn[sg], 1u);
          if (p < SF_CAP) {
            buf[2 * p] = hi;
            buf[2 * p + 1] = lo;
          } else {
            atomicOr(err, ERR_INVARIANT);
          }
        }
      }
      tot = warp_sum_u128(tot);
      above = warp_sum_u128(above);
      if (lane == 0) {
        sm.part[0][warp] = tot;
        sm.part[1][warp] = above;
      }
      __syncthreads();
      if (tid == 0) {
        u128 t = 0, a = 0;
        for (int w = 0; w < SS_BLOCK / 32; ++w) {
          t += sm.part[0][w];
          a += sm.part[1][w];
        }
        if (t) atomic_add_u128(&g_sum[4 * sg], &g_sum[4 * sg + 1], t);
        if (a) atomic_add_u128(&g_sum[4 * sg + 2], &g_sum[4 * sg + 3], a);
      }
    }
    __syncthreads();
    i0 = i1;
  }
}

__global__ void __launch_bounds__(SS_BLOCK) k_segsel_hist(const uint64_t* __restrict__ probs,
                                                          const uint64_t* __restrict__ keys,
                                                          const uint16_t* __restrict__ seg,
                                                          const uint64_t* __restrict__ n_dev,
                                                          const SegSel* __restrict__ sel,
                                                          uint32_t* __restrict__ g_cnt, uint64_t* __restrict__ g_sum,
                                                          uint64_t* __restrict__ g_buf, uint32_t* __restrict__ g_bufn,
                                                          uint32_t* err) {
  __shared__ SegHistSmem sm;
  segsel_hist_chunk(probs, keys, seg, n_dev, sel, g_cnt, g_sum, g_buf, g_bufn, err, blockIdx.x, gridDim.x, sm);
}

// One block per counting segment: pick the bin holding the target rank.
struct SegPickSmem {
  uint64_t w_c[8];
  uint32_t first;
};

// Slot `slot` (blockDim.x == 256).
__device__ __forceinline__ void segsel_pick_slot(SegSel* __restrict__ sel, const uint32_t* __restrict__ g_cnt,
                                                 uint32_t slot, SegPickSmem& sm) {
  SegSel& st = sel[slot];
  if (!st.active || st.done || seg_collects(st)) return;
  const uint32_t* cnt = g_cnt + (uint64_t)slot * SS_BINS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bits = (int)st.bits;
  int D, shift;
  sel_digit(bits, &D, &shift);
  const int nbins = 1 << D;
  const int per = (nbins + 255) / 256;
  const int b0 = tid * per;
  uint64_t my_c = 0;
  for (int b = b0; b < b0 + per && b < nbins; ++b) my_c += cnt[b];
  uint64_t xc = my_c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t yc = __shfl_up_sync(0xffffffffu, (unsigned long long)xc, o);
    if (lane >= o) xc += yc;
  }
  if (lane == 31) sm.w_c[warp] = xc;
  if (tid == 0) sm.first = 0xffffffffu;
  __syncthreads();
  uint64_t base_c = 0;
  for (int w = 0; w < warp; ++w) base_c += sm.w_c[w];
  const uint64_t excl_c = base_c + xc - my_c;
  const uint64_t target = st.target;
  const uint64_t before_c = st.before_count;
  {
    uint64_t cc = before_c + excl_c;
    for (int b = b0; b < b0 + per && b < nbins; ++b) {
      const uint32_t c = cnt[b];
      cc += c;
      if (c > 0 && cc >= target) {
        atomicMin(&sm.first, (uint32_t)b);
        break;
      }
    }
  }
  __syncthreads();
  const uint32_t first = sm.first;
  if (first == 0xffffffffu) {
    if (tid == 0) st.done = 2;  // fewer terms than the target: not reached for an active segment
    return;
  }
  if ((int)first >= b0 && (int)first < b0 + per) {
    uint64_t bc = before_c + excl_c;
    for (int b = b0; b < (int)first; ++b) bc += cnt[b];
    u128 prefix = make_u128(st.prefix_hi, st.prefix_lo);
    prefix |= ((u128)first) << shift;
    st.prefix_hi = (uint64_t)(prefix >> 64);
    st.prefix_lo = (uint64_t)prefix;
    st.bits = (uint32_t)(bits + D);
    st.before_count = bc;
    st.bin_count = cnt[first];  // at 128 bits a single term: collected next
  }
}

__global__ void __launch_bounds__(256) k_segsel_pick(SegSel* __restrict__ sel, const uint32_t* __restrict__ g_cnt) {
  __shared__ SegPickSmem sm;
  segsel_pick_slot(sel, g_cnt, blockIdx.x, sm);
}

// cfg picks the scan's blocks per SM: 2, 4 or 8.
void launch_segsel_level(const uint64_t* probs, const uint64_t* keys, const uint16_t* seg, const uint64_t* n_dev,
                         SegSel* sel, int slots, uint32_t* g_cnt, uint64_t* g_sum, uint64_t* g_buf, uint32_t* g_bufn,
                         uint32_t* err, int cfg, cudaStream_t st) {
  cudaMemsetAsync(g_cnt, 0, sizeof(uint32_t) * SS_BINS * slots, st);
  cudaMemsetAsync(g_sum, 0, sizeof(uint64_t) * 4 * slots, st);
  cudaMemsetAsync(g_bufn, 0, sizeof(uint32_t) * slots, st);
  const unsigned grid = 148u * (2u << (cfg < 0 ? 0 : (cfg > 2 ? 2 : cfg)));
  k_segsel_hist<<<grid, SS_BLOCK, 0, st>>>(probs, keys, seg, n_dev, sel, g_cnt, g_sum, g_buf, g_bufn, err);
  k_segsel_pick<<<slots, 256, 0, st>>>(sel, g_cnt);
}

void launch_segsel_pick(SegSel* sel, int slots, const uint32_t* g_cnt, cudaStream_t st) {
  k_segsel_pick<<<slots, 256, 0, st>>>(sel, g_cnt);
}

// Select state of every slot for this step: a slot in use with more terms
// than its K is truncated to its top K (Sec. III).
__device__ __forceinline__ void segsel_init_slot(SegSel* __restrict__ sel, const SegGate* __restrict__ gates,
                                                 const uint64_t* __restrict__ start, const uint64_t* __restrict__ end,
                                                 int s) {
  SegSel st;
  memset(&st, 0, sizeof(SegSel));
  const uint64_t count = end[s] > start[s] ? end[s] - start[s] : 0;
  const SegGate& g = gates[s];
  if (g.m >= 0 && g.K > 0 && count > g.K) {
    st.active = 1;
    st.bits = 1;
    st.prefix_hi = 1ull << 63;
    st.target = g.K;
    st.bin_count = count;  // a small segment is copied whole by the first scan
  }
  sel[s] = st;
}

__global__ void k_segsel_init(SegSel* __restrict__ sel, const SegGate* __restrict__ gates,
                              const uint64_t* __restrict__ start, const uint64_t* __restrict__ end, int slots) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= slots) return;
  segsel_init_slot(sel, gates, start, end, s);
}

void launch_segsel_init(SegSel* sel, const SegGate* gates, const uint64_t* start, const uint64_t* end, int slots,
                        cudaStream_t st) {
  k_segsel_init<<<(slots + 127) / 128, 128, 0, st>>>(sel, gates, start, end, slots);
}

// Finish: one block per segment collected in this level's scan resolves the
// cut among the copied terms, level after level inside shared memory.
struct SegFinishSmem {
  uint32_t cnt[SS_BINS];
  uint64_t mass[2 * SS_BINS];
  uint64_t w_c[8];
  u128 w_m[8];
  uint32_t first;
  SegSel st;  // the segment's select state, updated here and written back once
};

// Slot `slot` (blockDim.x == 256).  With STAGE the copied terms are first
// staged in shared memory (stage: 2 * SF_CAP words); without, every level
// reads them from the copy buffer in global memory (a few KB, L2-resident).
template <bool STAGE>
__device__ __forceinline__ void segsel_finish_slot(const uint64_t* __restrict__ g_buf,
                                                   const uint32_t* __restrict__ g_bufn,
                                                   const uint64_t* __restrict__ g_sum, SegSel* sel, uint32_t* err,
                                                   uint32_t slot, SegFinishSmem& sm, uint64_t* stage) {
  SegSel& st = sm.st;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    st = sel[slot];
  }
  __syncthreads();
  // only segments whose terms this level's scan copied (a collected bin is
  // never empty; a segment that entered collect mode in this level's pick
  // has nothing copied yet and waits for the next scan)
  const uint32_t copied = g_bufn[slot];
  if (!st.active || st.done || copied == 0) return;
  const uint32_t nb = copied < SF_CAP ? copied : SF_CAP;
  if (tid == 0) {
    st.total_mass_hi = g_sum[4 * slot];
    st.total_mass_lo = g_sum[4 * slot + 1];
    st.before_mass_hi = g_sum[4 * slot + 2];
    st.before_mass_lo = g_sum[4 * slot + 3];
  }
  const uint64_t* buf = g_buf + (uint64_t)slot * 2 * SF_CAP;
  const uint64_t* bz = buf;  // term i: (bz[2 i], bz[2 i + 1]) = (hi, lo)
  if (STAGE) {
    for (uint32_t i = tid; i < nb; i += blockDim.x) {
      stage[2 * i] = buf[2 * i];
      stage[2 * i + 1] = buf[2 * i + 1];
    }
    bz = stage;
  }
  __syncthreads();
  for (int it = 0; it < 128; ++it) {
    __syncthreads();
    if (st.done) break;
    const int bits = (int)st.bits;
    if (st.bin_count == 1) {
      // one term left under the prefix: it is the cut, the terms before it
      // are those counted so far (or the target is never reached)
      for (uint32_t i = tid; i < nb; i += blockDim.x) {
        if (!z_matches(bz[2 * i], bz[2 * i + 1], st.prefix_hi, st.prefix_lo, bits)) continue;
        const uint64_t cc = st.before_count + 1;
        if (cc < st.target) {
          st.done = 2;
          continue;
        }
        const uint64_t pbits = ~bz[2 * i];
        const u128 sc = make_u128(st.before_mass_hi, st.before_mass_lo) + fx_from_bits(pbits, err);
        st.cut_pbits = pbits;
        st.cut_key = bz[2 * i + 1];
        st.cut_count = cc;
        st.cut_mass_hi = (uint64_t)(sc >> 64);
        st.cut_mass_lo = (uint64_t)sc;
        st.done = 1;
      }
      __syncthreads();
      if (st.done) break;
    }
    int D, shift;
    sel_digit(bits, &D, &shift);
    for (int b = tid; b < SS_BINS; b += blockDim.x) {
      sm.cnt[b] = 0;
      sm.mass[2 * b] = sm.mass[2 * b + 1] = 0;
    }
    if (tid == 0) sm.first = 0xffffffffu;
    __syncthreads();
    for (uint32_t i = tid; i < nb; i += blockDim.x) {
      if (!z_matches(bz[2 * i], bz[2 * i + 1], st.prefix_hi, st.prefix_lo, bits)) continue;
      const uint32_t dg = (uint32_t)(make_u128(bz[2 * i], bz[2 * i + 1]) >> shift) & ((1u << D) - 1u);
      atomicAdd(&sm.cnt[dg], 1u);
      atomic_add_u128(&sm.mass[2 * dg], &sm.mass[2 * dg + 1], fx_from_bits(~bz[2 * i], err));
    }
    __syncthreads();
    const int nbins = 1 << D;
    const int per = (nbins + 255) / 256;
    const int b0 = tid * per;
    uint64_t my_c = 0;
    u128 my_m = 0;
    for (int b = b0; b < b0 + per && b < nbins; ++b) {
      my_c += sm.cnt[b];
      my_m += make_u128(sm.mass[2 * b], sm.mass[2 * b + 1]);
    }
    uint64_t xc = my_c;
    u128 xm = my_m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t yc = __shfl_up_sync(0xffffffffu, (unsigned long long)xc, o);
      const uint64_t yh = __shfl_up_sync(0xffffffffu, (unsigned long long)(xm >> 64), o);
      const uint64_t yl = __shfl_up_sync(0xffffffffu, (unsigned long long)(uint64_t)xm, o);
      if (lane >= o) {
        xc += yc;
        xm += make_u128(yh, yl);
      }
    }
    if (lane == 31) {
      sm.w_c[warp] = xc;
      sm.w_m[warp] = xm;
    }
    __syncthreads();
    uint64_t base_c = 0;
    u128 base_m = 0;
    for (int w = 0; w < warp; ++w) {
      base_c += sm.w_c[w];
      base_m += sm.w_m[w];
    }
    const uint64_t excl_c = base_c + xc - my_c;
    const u128 excl_m = base_m + xm - my_m;
    const uint64_t before_c = st.before_count;
    const u128 before_m = make_u128(st.before_mass_hi, st.before_mass_lo);
    const uint64_t target = st.target;
    {
      uint64_t cc = before_c + excl_c;
      for (int b = b0; b < b0 + per && b < nbins; ++b) {
        const uint32_t c = sm.cnt[b];
        cc += c;
        if (c > 0 && cc >= target) {
          atomicMin(&sm.first, (uint32_t)b);
          break;
        }
      }
    }
    __syncthreads();
    const uint32_t first = sm.first;
    if (first == 0xffffffffu) {
      if (tid == 0) st.done = 2;
      __syncthreads();
      break;
    }
    if ((int)first >= b0 && (int)first < b0 + per) {
      uint64_t bc = before_c + excl_c;
      u128 bm = before_m + excl_m;
      for (int b = b0; b < (int)first; ++b) {
        bc += sm.cnt[b];
        bm += make_u128(sm.mass[2 * b], sm.mass[2 * b + 1]);
      }
      u128 prefix = make_u128(st.prefix_hi, st.prefix_lo);
      prefix |= ((u128)first) << shift;
      const int nbits = bits + D;
      st.prefix_hi = (uint64_t)(prefix >> 64);
      st.prefix_lo = (uint64_t)prefix;
      st.bits = (uint32_t)nbits;
      st.before_count = bc;
      st.before_mass_hi = (uint64_t)(bm >> 64);
      st.before_mass_lo = (uint64_t)bm;
      st.bin_count = sm.cnt[first];
      if (nbits == 128) {
        const uint64_t pbits = ~(uint64_t)(prefix >> 64);
        const u128 sc = bm + fx_from_bits(pbits, err);
        st.cut_pbits = pbits;
        st.cut_key = (uint64_t)prefix;
        st.cut_count = bc + 1;
        st.cut_mass_hi = (uint64_t)(sc >> 64);
        st.cut_mass_lo = (uint64_t)sc;
        st.done = 1;
      }
    }
  }
  __syncthreads();
  if (tid == 0) sel[slot] = st;
}

__global__ void __launch_bounds__(256) k_segsel_finish(const uint64_t* __restrict__ g_buf,
                                                       const uint32_t* __restrict__ g_bufn,
                                                       const uint64_t* __restrict__ g_sum, SegSel* sel,
                                                       uint32_t* err) {
  extern __shared__ __align__(16) uint64_t s_stage[];
  __shared__ SegFinishSmem sm;
  segsel_finish_slot<true>(g_buf, g_bufn, g_sum, sel, err, blockIdx.x, sm, s_stage);
}

cudaError_t layer_attrs();

// Kernel attributes (dynamic shared memory) set once, outside any stream
// capture.
cudaError_t batch_prepare() {
  static DeviceOnce once;
  cudaError_t e = once.run([] {
    cudaError_t r = cudaFuncSetAttribute(k_segsel_finish, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * sizeof(uint64_t) * SF_CAP));
    if (r == cudaSuccess) r = seg_apply_attrs<double>();
    if (r == cudaSuccess) r = seg_apply_attrs<float>();
    if (r == cudaSuccess) r = layer_attrs();
    return r;
  });
  if (e == cudaSuccess) e = sort_prepare();
  return e == cudaSuccess ? regroup_prepare() : e;  // the step groups with the partition and merge kernels
}

void launch_segsel_finish(const uint64_t* g_buf, const uint32_t* g_bufn, const uint64_t* g_sum, SegSel* sel,
                          int slots, uint32_t* err, cudaStream_t st) {
  const size_t smem = 2 * sizeof(uint64_t) * SF_CAP;
  (void)batch_prepare();  // checked at the batch's creation; a launch without it fails loudly
  k_segsel_finish<<<slots, 256, smem, st>>>(g_buf, g_bufn, g_sum, sel, err);
}

// Renormalisation scale of every segment that found a cut.
__device__ __forceinline__ void segsel_scale_slot(SegSel& st) {
  if (st.active && st.done == 1) st.scale = __ddiv_rn(1.0, __dsqrt_rn(fx_to_double(make_u128(st.cut_mass_hi, st.cut_mass_lo))));
}

__global__ void k_segsel_scale(SegSel* sel, int slots) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= slots) return;
  segsel_scale_slot(sel[s]);
}

void launch_segsel_scale(SegSel* sel, int slots, cudaStream_t st) {
  k_segsel_scale<<<(slots + 127) / 128, 128, 0, st>>>(sel, slots);
}

// ---------------------------------------------------------------- compaction
constexpr int SC_BLOCK = 256, SC_ITEMS = 8;

// Keep, in each segment with a cut, the terms not after its cut (scaled);
// other segments keep everything unchanged.
struct SegTruncSmem {
  CompactShared<SC_BLOCK> cs;
  uint64_t tile;
  uint16_t list[SC_BLOCK * SC_ITEMS];
  uint16_t slots[SC_BLOCK * SC_ITEMS];  // slot of each kept term (segment bounds)
};

// Tiles taken from ctl->tile_counter[2] until none is left; the kept count
// lands in ctl->count[2].
template <typename C2>
__device__ __forceinline__ void seg_truncate_run(
    const uint64_t* __restrict__ keys, const C2* __restrict__ amps, const uint64_t* __restrict__ probs,
    const uint16_t* __restrict__ seg, const uint64_t* __restrict__ n_dev, uint64_t n_max,
    const SegSel* __restrict__ sel, uint64_t* __restrict__ keys_out, C2* __restrict__ amps_out,
    uint16_t* __restrict__ seg_out, uint64_t* __restrict__ start, uint64_t* __restrict__ end, uint64_t* lookback,
    Ctl* ctl, SegTruncSmem& sm) {
  typedef TileLayout<SC_BLOCK, SC_ITEMS> L;
  const uint64_t n = *n_dev;
  if (n > n_max) {  // the look-back buffer was sized for n_max terms
    if (threadIdx.x == 0) atomicOr(&ctl->err, ERR_INVARIANT);
    return;
  }
  const uint64_t tiles = (n + L::TILE - 1) / L::TILE;
  while (true) {
    if (threadIdx.x == 0) sm.tile = atomicAdd((unsigned long long*)&ctl->tile_counter[2], 1ull);
    __syncthreads();
    const uint64_t tile = sm.tile;
    if (tile >= tiles) break;
    const uint64_t base = tile * L::TILE;
    bool flag[SC_ITEMS];
    uint32_t pos[SC_ITEMS];
    uint16_t sgv[SC_ITEMS];
    uint64_t pbv[SC_ITEMS];
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
      const uint64_t i = L::index(base, j);
      sgv[j] = i < n ? seg[i] : (uint16_t)0;
      pbv[j] = i < n ? probs[i] : 0ull;
    }
    // a segment's cut, cached across a thread's items (a tile rarely spans
    // more than one segment)
    int last = -1;
    bool cut_on = false;
    uint64_t cut_pb = 0, cut_key = 0;
    double scale = 1.0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
      const uint64_t i = L::index(base, j);
      bool f = false;
      if (i < n) {
        if ((int)sgv[j] != last) {
          last = sgv[j];
          const SegSel& st = sel[last];
          cut_on = st.active && st.done == 1;
          cut_pb = st.cut_pbits;
          cut_key = st.cut_key;
          scale = st.scale;
        }
        f = !cut_on || pbv[j] > cut_pb || (pbv[j] == cut_pb && keys[i] <= cut_key);
      }
      flag[j] = f;
    }
    tile_compact<SC_BLOCK, SC_ITEMS>(flag, pos, sm.cs, lookback, tile, &ctl->err);
    // list the kept terms, then process the list densely (all lanes busy,
    // contiguous writes)
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j)
      if (flag[j]) sm.list[pos[j]] = (uint16_t)(L::index(base, j) - base);
    __syncthreads();
    last = -1;
    const uint32_t kept = sm.cs.tile_total;
    const uint64_t ob = sm.cs.tile_base_out;
    for (uint32_t t = threadIdx.x; t < kept; t += SC_BLOCK) {
      const uint64_t i = base + sm.list[t];
      const uint16_t sg = seg[i];
      if ((int)sg != last) {
        last = sg;
        const SegSel& st = sel[last];
        cut_on = st.active && st.done == 1;
        scale = st.scale;
      }
      C2 a = amps[i];
      if (cut_on) a = amp_scaled(a, scale);
      keys_out[ob + t] = keys[i];
      amps_out[ob + t] = a;
      seg_out[ob + t] = sg;
      sm.slots[t] = sg;
    }
    if (start) {
      __syncthreads();
      for (uint32_t t = threadIdx.x; t < kept; t += SC_BLOCK) seg_bound_marks(sm.slots, t, kept, ob, start, end);
    }
    if (tile == tiles - 1 && threadIdx.x == 0) ctl->count[2] = sm.cs.tile_base_out + sm.cs.tile_total;
    __syncthreads();
  }
}

template <typename C2>
__global__ void __launch_bounds__(SC_BLOCK, 4) k_seg_truncate(
    const uint64_t* __restrict__ keys, const C2* __restrict__ amps, const uint64_t* __restrict__ probs,
    const uint16_t* __restrict__ seg, const uint64_t* __restrict__ n_dev, uint64_t n_max,
    const SegSel* __restrict__ sel, uint64_t* __restrict__ keys_out, C2* __restrict__ amps_out,
    uint16_t* __restrict__ seg_out, uint64_t* __restrict__ start, uint64_t* __restrict__ end, uint64_t* lookback,
    Ctl* ctl) {
  __shared__ SegTruncSmem sm;
  seg_truncate_run<C2>(keys, amps, probs, seg, n_dev, n_max, sel, keys_out, amps_out, seg_out, start, end, lookback,
                       ctl, sm);
}

void launch_seg_truncate(int prec, const uint64_t* keys, const void* amps, const uint64_t* probs, const uint16_t* seg,
                         const uint64_t* n_dev, uint64_t n_max, const SegSel* sel, uint64_t* keys_out,
                         void* amps_out, uint16_t* seg_out, uint64_t* start, uint64_t* end, uint64_t* lookback,
                         Ctl* ctl, int cfg, cudaStream_t st) {
  const uint64_t tiles = (n_max + SC_BLOCK * SC_ITEMS - 1) / (SC_BLOCK * SC_ITEMS);
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * (tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[2], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[2], 0, sizeof(uint64_t), st);
  if (n_max == 0) return;
  // cfg picks the persistent blocks per SM: 4 or 8
  const uint64_t per_sm = cfg == 0 ? 4 : 8;
  const uint64_t grid = tiles < 148 * per_sm ? tiles : 148 * per_sm;
  if (prec == 0)
    k_seg_truncate<double2><<<(unsigned)grid, SC_BLOCK, 0, st>>>(keys, (const double2*)amps, probs, seg, n_dev, n_max,
                                                                 sel, keys_out, (double2*)amps_out, seg_out,
                                                                 start, end, lookback, ctl);
  else
    k_seg_truncate<float2><<<(unsigned)grid, SC_BLOCK, 0, st>>>(keys, (const float2*)amps, probs, seg, n_dev, n_max,
                                                                sel, keys_out, (float2*)amps_out, seg_out,
                                                                start, end, lookback, ctl);
}

// ---------------------------------------------------------------- one launch per layer
// The whole step of the batched form as one persistent kernel: a grid of
// co-resident blocks (cooperative launch) runs the phases of the step one
// after another, with a grid-wide barrier between phases, and every size
// is read on the device (the term counts of the previous phase), so the
// launch and the copies around it are captured once in a CUDA graph and
// replayed for every later step of the same shape.  The phases are the
// bodies of the standalone kernels above and of the regrouping kernels,
// with 256-thread blocks: the sort keys; the stable partition by the gate
// bits and the merge levels; group heads; the mat-vec (which also counts the
// select's first digit per slot); segment bounds; the per-slot top-k select
// level after level until every cut is found; the renormalisation scales;
// the compaction and the new bounds.

constexpr int LAYER_THREADS = 256;
constexpr int LAYER_ITEMS = RG_TILE / LAYER_THREADS;  // partition and merge items per thread
constexpr int LAYER_LEVELS = 16;                       // select levels before a cut counts as unresolved
constexpr int LAYER_GPT = 1;                           // mat-vec groups per thread
constexpr size_t LAYER_HDR = (sizeof(SegApplySmem) > sizeof(MergeHdr) ? sizeof(SegApplySmem) : sizeof(MergeHdr)) /
                                 128 * 128 + 128;

// Spin limit of the grid barrier (polls with back-off up to 1 us: a few
// seconds); a block that gives up records ERR_TIMEOUT and the layer stops.
constexpr uint32_t LAYER_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of the layer kernel (all threads of every block call
// it).  The last block to arrive reads the error word (every error recorded
// before the barrier is visible to it) and publishes the next generation
// with a stop bit, so all blocks leave the barrier with the same decision.
// Returns true when the layer must stop.
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The first block charges the time since the last barrier to `phase`.
__device__ __forceinline__ void layer_phase_mark(LayerCtl* lc, int phase) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const uint64_t now = global_ns();
    lc->phase_ns[phase] += now - lc->t_last;
    lc->t_last = now;
  }
}

__device__ __forceinline__ bool layer_sync(LayerCtl* lc, uint32_t nblocks, uint32_t* err, int phase) {
  __syncthreads();
  int stop = 0;
  if (threadIdx.x == 0) {
    const uint32_t g0 = ld_acquire_u32(&lc->bar_gen) & 0x7fffffffu;
    __threadfence();
    const uint32_t arrived = atomicAdd(&lc->bar_count, 1u) + 1u;
    __threadfence();
    if (arrived == nblocks) {
      const uint32_t e = ld_acquire_u32(err);
      atomicExch(&lc->bar_count, 0u);
      __threadfence();
      st_release_u32(&lc->bar_gen, ((g0 + 1u) & 0x7fffffffu) | (e ? 0x80000000u : 0u));
      stop = e != 0;
    } else {
      uint32_t spins = 0, ns = 32;
      while (true) {
        const uint32_t g = ld_acquire_u32(&lc->bar_gen);
        if ((g & 0x7fffffffu) != g0) {
          stop = (int)(g >> 31);
          break;
        }
        if (++spins > LAYER_SPIN_LIMIT) {
          atomicOr(err, ERR_TIMEOUT);
          stop = 1;
          break;
        }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
      }
    }
    __threadfence();
  }
  layer_phase_mark(lc, phase);
  return __syncthreads_or(stop) != 0;
}

template <typename T>
__device__ __forceinline__ T& smem_as(uint8_t* p) {
  return *reinterpret_cast<T*>(p);
}

template <typename Real, int MAXD>
__global__ void __launch_bounds__(LAYER_THREADS, MAXD <= 4 ? 4 : (MAXD == 8 ? 2 : 1)) k_seg_layer(const LayerParams P) {
  typedef typename SCplx<Real>::T C2;
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* const dyn = smem + LAYER_HDR;  // a phase's staging area, after its shared variables
  const uint32_t cta = blockIdx.x, ncta = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint64_t gtid = (uint64_t)cta * LAYER_THREADS + tid, gstride = (uint64_t)ncta * LAYER_THREADS;
  const LayerStep S = *P.step;
  const int shift = S.shift, top = S.top, m = S.m, D = 1 << m;
  Ctl* ctl = P.ctl;
  uint32_t* err = &ctl->err;
  LayerCtl* lc = P.lc;
  // the state's buffer set and term count (rewritten only at the very end)
  const int cin = (int)lc->cur, cmv = 1 - cin;
  const uint64_t N = lc->n_cur;
  const uint64_t* keys_in = P.keys[cin];
  const uint16_t* seg_in = P.seg[cin];
  const C2* amps_in = (const C2*)P.amps[cin];
  uint64_t* keys_mv = P.keys[cmv];
  C2* amps_mv = (C2*)P.amps[cmv];
  uint64_t* probs_mv = P.probs[cmv];
  uint16_t* seg_mv = P.seg[cmv];
  uint64_t* lb_heads = P.lb;
  uint64_t* lb_apply = lb_heads + P.lb_heads_words;
  uint64_t* lb_trunc = lb_apply + P.lb_apply_words;

  // clear this layer's counters, look-backs and select histograms; tables
  for (uint64_t i = gtid; i < P.lb_heads_words + P.lb_apply_words + P.lb_trunc_words; i += gstride) P.lb[i] = 0;
  for (uint64_t i = gtid; i < (uint64_t)top * SEL_BINS; i += gstride) P.sel_cnt[0][i] = P.sel_cnt[1][i] = 0;
  for (uint64_t i = gtid; i < (uint64_t)top; i += gstride) {
    P.sel_bufn[0][i] = P.sel_bufn[1][i] = 0;
    P.start[i] = P.start_tr[i] = ~0ull;
    P.end[i] = P.end_tr[i] = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) P.sel_mass[0][4 * i + j] = P.sel_mass[1][4 * i + j] = 0;
  }
  if (gtid < 16) P.hist16[gtid] = 0;
  if (gtid == 0) {
    for (int j = 0; j < 3; ++j) {
      ctl->tile_counter[j] = 0;
      ctl->count[j] = 0;
    }
    lc->truncated = 0;
    lc->unresolved = 0;
  }
  if (cta == 0 && tid == 0) lc->t_last = global_ns();  // phase times add up over the steps
  for (uint32_t vb = cta; vb < (uint32_t)top; vb += ncta) {
    seg_tables_slot(P.gates, P.tables, vb, smem_as<SegTablesSmem>(smem));
    __syncthreads();
  }
  if (layer_sync(lc, ncta, err, LP_SETUP)) return;

  // sort keys, then the grouping: partition by the gate bits, m merge levels
  seg_keys_range(keys_in, seg_in, N, P.gates, P.tables, shift, P.sk[1], gtid, gstride);
  if (layer_sync(lc, ncta, err, LP_KEYS)) return;
  GateParams gp;
  memset(&gp, 0, sizeof(gp));
  gp.m = m;
  gp.direct = 1;
  const uint64_t tiles = (N + RG_TILE - 1) / RG_TILE;
  uint32_t* cnt = P.part;
  uint32_t* off = cnt + (uint64_t)D * tiles;
  for (uint64_t t = cta; t < tiles; t += ncta) {
    part_counts_tile<LAYER_THREADS, LAYER_ITEMS>(P.sk[1], N, gp, tiles, cnt, P.hist16, t,
                                                 smem_as<PartCountsSmem>(smem));
    __syncthreads();
  }
  if (layer_sync(lc, ncta, err, LP_COUNTS)) return;
  uint64_t nkeep = 0;  // terms of the slots that stay (a removed slot's terms are left out)
  for (int d = 0; d < D; ++d) nkeep += P.hist16[d];
  for (uint32_t d = cta; d < (uint32_t)D; d += ncta) {
    tile_offsets_digit<LAYER_THREADS>(cnt, P.hist16, tiles, off, (int)d, smem_as<TileOffsetsSmem<LAYER_THREADS>>(smem));
    __syncthreads();
  }
  if (layer_sync(lc, ncta, err, LP_OFFSETS)) return;
  for (uint64_t t = cta; t < tiles; t += ncta) {
    part_scatter_tile<LAYER_THREADS, LAYER_ITEMS, true>(P.sk[1], N, gp, tiles, off, P.sk[0], P.sidx[0], t,
                                                        smem_as<PartScatterSmem<LAYER_THREADS>>(smem));
    __syncthreads();
  }
  if (layer_sync(lc, ncta, err, LP_SCATTER)) return;
  int cur = 0;
  const uint32_t mblocks = (uint32_t)((N + MG_TILE - 1) / MG_TILE) + (uint32_t)D;
  uint32_t* splits = cnt;  // the partition's counts are no longer needed
  for (int level = 1; level <= m; ++level) {
    for (uint64_t w = gtid >> 5; w < mblocks; w += gstride >> 5)
      merge_split_warp(P.sk[cur], P.hist16, D, level, (uint32_t)w, splits, lane);
    if (layer_sync(lc, ncta, err, LP_SPLITS)) return;
    for (uint32_t b = cta; b < mblocks; b += ncta) {
      merge_tile<LAYER_THREADS, LAYER_ITEMS, true>(P.sk[cur], P.sidx[cur], P.sk[1 - cur], P.sidx[1 - cur],
                                                   P.hist16, D, level, splits, b, smem_as<MergeHdr>(smem), dyn);
      __syncthreads();
    }
    if (layer_sync(lc, ncta, err, LP_MERGE)) return;
    cur ^= 1;
  }

  // group heads, then the mat-vec (counting the select's first digit)
  seg_heads_run(P.sk[cur], nkeep, shift, P.gates, P.rank_slot, P.heads, lb_heads, ctl, smem_as<SegHeadsSmem>(smem));
  if (layer_sync(lc, ncta, err, LP_HEADS)) return;
  if (tid == 0) smem_as<SegApplySmem>(smem).hcnt = reinterpret_cast<uint32_t*>(dyn + seg_apply_smem<C2>(MAXD, LAYER_GPT));
  __syncthreads();
  seg_apply_run<Real, MAXD, LAYER_GPT>(P.sk[cur], P.sidx[cur], nkeep, P.heads, amps_in, shift, P.gates,
                                       P.rank_slot, keys_in, keys_mv, amps_mv, probs_mv, seg_mv,
                                       P.sel_cnt[0], P.start, P.end, lb_apply, P.lb_apply_words - 1, ctl,
                                       smem_as<SegApplySmem>(smem), dyn);
  if (layer_sync(lc, ncta, err, LP_APPLY)) return;

  // per-slot top-k: bounds, select state, the first level's pick, then
  // scan / pick / finish levels until every active slot's cut is found
  for (uint64_t s = gtid; s < (uint64_t)top; s += gstride) segsel_init_slot(P.sel, P.gates, P.start, P.end, (int)s);
  if (layer_sync(lc, ncta, err, LP_INIT)) return;
  for (uint32_t vb = cta; vb < (uint32_t)top; vb += ncta) {
    segsel_pick_slot(P.sel, P.sel_cnt[0], vb, smem_as<SegPickSmem>(smem));
    __syncthreads();
  }
  if (layer_sync(lc, ncta, err, LP_PICK1)) return;
  int par = 1;
  bool pending = true;
  for (int level = 0; level < LAYER_LEVELS && pending; ++level) {
    // the other parity's histograms were read by the previous level: clear them for the next
    for (uint64_t i = gtid; i < (uint64_t)top * SEL_BINS; i += gstride) P.sel_cnt[1 - par][i] = 0;
    for (uint64_t i = gtid; i < (uint64_t)top; i += gstride) {
      P.sel_bufn[1 - par][i] = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) P.sel_mass[1 - par][4 * i + j] = 0;
    }
    segsel_hist_chunk(probs_mv, keys_mv, seg_mv, &ctl->count[1], P.sel, P.sel_cnt[par], P.sel_mass[par],
                      P.sel_buf, P.sel_bufn[par], err, cta, ncta, smem_as<SegHistSmem>(smem));
    if (layer_sync(lc, ncta, err, LP_HIST)) return;
    for (uint32_t vb = cta; vb < (uint32_t)top; vb += ncta) {
      segsel_pick_slot(P.sel, P.sel_cnt[par], vb, smem_as<SegPickSmem>(smem));
      __syncthreads();
    }
    if (layer_sync(lc, ncta, err, LP_PICK)) return;
    for (uint32_t vb = cta; vb < (uint32_t)top; vb += ncta) {
      segsel_finish_slot<false>(P.sel_buf, P.sel_bufn[par], P.sel_mass[par], P.sel, err, vb,
                                smem_as<SegFinishSmem>(smem), nullptr);
      __syncthreads();
    }
    if (layer_sync(lc, ncta, err, LP_FINISH)) return;
    bool open = false;  // every block reads the same select states
    for (int s = tid; s < top; s += LAYER_THREADS) open |= P.sel[s].active && !P.sel[s].done;
    pending = __syncthreads_or(open) != 0;
    par ^= 1;
  }
  if (pending) {
    if (gtid == 0) {
      lc->unresolved = 1;
      atomicOr(err, ERR_INVARIANT);
    }
    return;
  }
  for (uint64_t s = gtid; s < (uint64_t)top; s += gstride) {
    SegSel& st = P.sel[s];
    segsel_scale_slot(st);
    if (st.active && st.done == 1)  // retained mass F *= S_c / S_N (Sec. III)
      P.F[s] = __dmul_rn(P.F[s], __ddiv_rn(fx_to_double(make_u128(st.cut_mass_hi, st.cut_mass_lo)),
                                           fx_to_double(make_u128(st.total_mass_hi, st.total_mass_lo))));
  }
  bool cut = false;
  for (int s = tid; s < top; s += LAYER_THREADS) cut |= P.sel[s].active && P.sel[s].done == 1;
  const bool any_cut = __syncthreads_or(cut) != 0;
  if (layer_sync(lc, ncta, err, LP_SCALE)) return;
  if (!any_cut) {
    if (gtid == 0) {
      lc->cur = (uint32_t)cmv;
      lc->n_cur = ctl->count[1];
    }
    return;
  }

  // compaction of the cut slots, then their new bounds (a slot keeps at
  // least one term, so every bound written by the mat-vec is overwritten)
  const uint64_t n_max = (P.lb_trunc_words - 1) * (uint64_t)(SC_BLOCK * SC_ITEMS);
  seg_truncate_run<C2>(keys_mv, amps_mv, probs_mv, seg_mv, &ctl->count[1], n_max, P.sel, P.keys[cin],
                       (C2*)P.amps[cin], P.seg[cin], P.start_tr, P.end_tr, lb_trunc, ctl,
                       smem_as<SegTruncSmem>(smem));
  if (layer_sync(lc, ncta, err, LP_TRUNC)) return;
  if (gtid == 0) {
    lc->truncated = 1;
    lc->cur = (uint32_t)cin;
    lc->n_cur = ctl->count[2];
  }
}

template <typename Real, int MAXD>
constexpr size_t layer_smem() {
  typedef typename SCplx<Real>::T C2;
  size_t a = seg_apply_smem<C2>(MAXD, LAYER_GPT) + sizeof(uint32_t) * SEL_BINS, b = merge_smem_bytes(true),
         c = sizeof(SegFinishSmem);
  size_t x = a > b ? a : b;
  return LAYER_HDR + (x > c ? x : c);
}

template <typename Real, int MAXD>
cudaError_t layer_attr() {
  return cudaFuncSetAttribute(k_seg_layer<Real, MAXD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)layer_smem<Real, MAXD>());
}

template <typename Real, int MAXD>
cudaError_t layer_launch(const LayerParams& P, unsigned grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = LAYER_THREADS;
  cfg.dynamicSmemBytes = layer_smem<Real, MAXD>();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_seg_layer<Real, MAXD>, P);
}

template <typename Real, int MAXD>
cudaError_t layer_blocks(int* per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_seg_layer<Real, MAXD>, LAYER_THREADS,
                                                       layer_smem<Real, MAXD>());
}

static int layer_maxd(int m) { return m <= 1 ? 2 : (1 << m); }

cudaError_t seg_layer_grid(int prec, int m, int sms, unsigned* grid) {
  int per = 0;
  const int d = layer_maxd(m);
  cudaError_t e;
  if (prec == 0)
    e = d == 2 ? layer_blocks<double, 2>(&per) : d == 4 ? layer_blocks<double, 4>(&per)
        : d == 8 ? layer_blocks<double, 8>(&per) : layer_blocks<double, 16>(&per);
  else
    e = d == 2 ? layer_blocks<float, 2>(&per) : d == 4 ? layer_blocks<float, 4>(&per)
        : d == 8 ? layer_blocks<float, 8>(&per) : layer_blocks<float, 16>(&per);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  *grid = (unsigned)(per * sms);
  return cudaSuccess;
}

cudaError_t launch_seg_layer(int prec, int m, const LayerParams& P, unsigned grid, cudaStream_t st) {
  const int d = layer_maxd(m);
  if (prec == 0)
    return d == 2 ? layer_launch<double, 2>(P, grid, st) : d == 4 ? layer_launch<double, 4>(P, grid, st)
           : d == 8 ? layer_launch<double, 8>(P, grid, st) : layer_launch<double, 16>(P, grid, st);
  return d == 2 ? layer_launch<float, 2>(P, grid, st) : d == 4 ? layer_launch<float, 4>(P, grid, st)
         : d == 8 ? layer_launch<float, 8>(P, grid, st) : layer_launch<float, 16>(P, grid, st);
}

cudaError_t layer_attrs() {
  cudaError_t e = layer_attr<double, 2>();
  if (e == cudaSuccess) e = layer_attr<double, 4>();
  if (e == cudaSuccess) e = layer_attr<double, 8>();
  if (e == cudaSuccess) e = layer_attr<double, 16>();
  if (e == cudaSuccess) e = layer_attr<float, 2>();
  if (e == cudaSuccess) e = layer_attr<float, 4>();
  if (e == cudaSuccess) e = layer_attr<float, 8>();
  if (e == cudaSuccess) e = layer_attr<float, 16>();
  return e;
}

// ---------------------------------------------------------------- layer bookkeeping
__global__ void k_seg_append_layer(uint64_t* k0, uint64_t* k1, void* a0, void* a1, uint64_t* p0, uint64_t* p1,
                                   uint16_t* s0, uint16_t* s1, LayerCtl* lc, uint64_t* bounds, int max_slots,
                                   double* F, int slot, int prec) {
  const int cur = (int)lc->cur;
  const uint64_t at = lc->n_cur;
  uint64_t* keys = cur ? k1 : k0;
  void* amps = cur ? a1 : a0;
  uint64_t* probs = cur ? p1 : p0;
  uint16_t* seg = cur ? s1 : s0;
  keys[at] = 0;
  if (prec == 0) reinterpret_cast<double2*>(amps)[at] = make_double2(1.0, 0.0);
  else reinterpret_cast<float2*>(amps)[at] = make_float2(1.0f, 0.0f);
  probs[at] = 0x3ff0000000000000ull;
  seg[at] = (uint16_t)slot;
  const int pair = lc->truncated ? 2 : 0;  // the pair of bounds the last step left
  bounds[(uint64_t)pair * max_slots + slot] = at;
  bounds[(uint64_t)(pair + 1) * max_slots + slot] = at + 1;
  F[slot] = 1.0;
  lc->n_cur = at + 1;
}

void launch_seg_append_layer(uint64_t* const keys[2], void* const amps[2], uint64_t* const probs[2],
                             uint16_t* const seg[2], LayerCtl* lc, uint64_t* bounds, int max_slots, double* F,
                             int slot, int prec, cudaStream_t st) {
  k_seg_append_layer<<<1, 1, 0, st>>>(keys[0], keys[1], amps[0], amps[1], probs[0], probs[1], seg[0], seg[1], lc,
                                      bounds, max_slots, F, slot, prec);
}

// Peak of one slot: per block the canonical best (larger probability bits,
// then the smaller key) over a grid-stride share of the slot's range, then
// one block reduces the partials.
__device__ __forceinline__ bool peak_better(uint64_t pa, uint64_t ka, uint64_t pb, uint64_t kb) {
  return pa > pb || (pa == pb && ka < kb);
}

__device__ __forceinline__ void block_best(uint64_t& p, uint64_t& k, uint64_t* sp, uint64_t* sk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t op = __shfl_xor_sync(0xffffffffu, (unsigned long long)p, o);
    const uint64_t ok = __shfl_xor_sync(0xffffffffu, (unsigned long long)k, o);
    if (peak_better(op, ok, p, k)) {
      p = op;
      k = ok;
    }
  }
  if (lane == 0) {
    sp[warp] = p;
    sk[warp] = k;
  }
  __syncthreads();
  if (warp == 0) {
    p = lane < (int)(blockDim.x >> 5) ? sp[lane] : 0ull;
    k = lane < (int)(blockDim.x >> 5) ? sk[lane] : ~0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t op = __shfl_xor_sync(0xffffffffu, (unsigned long long)p, o);
      const uint64_t ok = __shfl_xor_sync(0xffffffffu, (unsigned long long)k, o);
      if (peak_better(op, ok, p, k)) {
        p = op;
        k = ok;
      }
    }
  }
}

__device__ __forceinline__ void seg_peak_range(const LayerCtl* lc, const uint64_t* bounds, int max_slots, int slot,
                                               int dev_range, uint64_t off, uint64_t count, int cur, uint64_t* a,
                                               uint64_t* e, int* c) {
  if (dev_range) {
    const int pair = lc->truncated ? 2 : 0;
    *a = bounds[(uint64_t)pair * max_slots + slot];
    *e = bounds[(uint64_t)(pair + 1) * max_slots + slot];
    *c = (int)lc->cur;
  } else {
    *a = off;
    *e = off + count;
    *c = cur;
  }
}

template <typename C2>
__global__ void __launch_bounds__(256) k_seg_peak_part(const uint64_t* k0, const uint64_t* k1, const C2* a0,
                                                       const C2* a1, int dev_range, const LayerCtl* lc,
                                                       const uint64_t* bounds, int max_slots, int slot, uint64_t off,
                                                       uint64_t count, int cur, uint64_t* part) {
  __shared__ uint64_t sp[8], sk[8];
  uint64_t a, e;
  int c;
  seg_peak_range(lc, bounds, max_slots, slot, dev_range, off, count, cur, &a, &e, &c);
  const uint64_t* keys = c ? k1 : k0;
  const C2* amps = c ? a1 : a0;
  uint64_t bp = 0, bk = ~0ull;
  for (uint64_t i = a + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < e; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t p = amp_prob_bits(amps[i]), k = keys[i];
    if (peak_better(p, k, bp, bk)) {
      bp = p;
      bk = k;
    }
  }
  block_best(bp, bk, sp, sk);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = bp;
    part[2 * blockIdx.x + 1] = bk;
  }
}

__global__ void __launch_bounds__(256) k_seg_peak_final(const uint64_t* part, int nparts, int dev_range,
                                                        const double* F, int slot, double F_host, uint64_t* out) {
  __shared__ uint64_t sp[8], sk[8];
  uint64_t bp = 0, bk = ~0ull;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x)
    if (peak_better(part[2 * i], part[2 * i + 1], bp, bk)) {
      bp = part[2 * i];
      bk = part[2 * i + 1];
    }
  block_best(bp, bk, sp, sk);
  if (threadIdx.x == 0) {
    out[0] = bk;
    out[1] = bp;
    const double f = dev_range ? F[slot] : F_host;
    out[2] = (uint64_t)__double_as_longlong(f);
  }
}

void launch_seg_peak(uint64_t* const keys[2], void* const amps[2], int prec, int dev_range, const LayerCtl* lc,
                     const uint64_t* bounds, int max_slots, const double* F, int slot, uint64_t off, uint64_t count,
                     int cur, double F_host, uint64_t* part, uint64_t* out, cudaStream_t st) {
  if (prec == 0)
    k_seg_peak_part<double2><<<PEAK_SEG_BLOCKS, 256, 0, st>>>(keys[0], keys[1], (const double2*)amps[0],
                                                             (const double2*)amps[1], dev_range, lc, bounds,
                                                             max_slots, slot, off, count, cur, part);
  else
    k_seg_peak_part<float2><<<PEAK_SEG_BLOCKS, 256, 0, st>>>(keys[0], keys[1], (const float2*)amps[0],
                                                            (const float2*)amps[1], dev_range, lc, bounds, max_slots,
                                                            slot, off, count, cur, part);
  k_seg_peak_final<<<1, 256, 0, st>>>(part, PEAK_SEG_BLOCKS, dev_range, F, slot, F_host, out);
}

// ---------------------------------------------------------------- new terms
__global__ void k_seg_append(uint64_t* keys, void* amps, uint64_t* probs, uint16_t* seg, uint64_t at, uint16_t slot,
                             int prec) {
  keys[at] = 0;
  if (prec == 0) reinterpret_cast<double2*>(amps)[at] = make_double2(1.0, 0.0);
  else reinterpret_cast<float2*>(amps)[at] = make_float2(1.0f, 0.0f);
  probs[at] = 0x3ff0000000000000ull;
  seg[at] = slot;
}

void launch_seg_append(uint64_t* keys, void* amps, uint64_t* probs, uint16_t* seg, uint64_t at, int slot, int prec,
                       cudaStream_t st) {
  k_seg_append<<<1, 1, 0, st>>>(keys, amps, probs, seg, at, (uint16_t)slot, prec);
}

}  // namespace sv
