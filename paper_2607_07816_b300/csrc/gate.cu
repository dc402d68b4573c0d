// Gate application: key transform, partner-group heads, per-group mat-vec.
//
// Sec. IV-A: every amplitude meets the column of U selected by its bits on
// the gate qubits; all amplitudes whose basis states agree outside those bits
// form one group, whose 2^m outputs are y[r'] = sum_r U[r'][r] x[r] (Eq. 3
// generalised).  Here the group is made contiguous by sorting on the key with
// the gate bits moved to the bottom (sk = squeeze(key) << m | r), so a group
// is a run of equal sk >> m with its members in ascending r.  One thread then
// computes one output (group, r') in registers, and zero outputs are dropped
// while the survivors are compacted in (group, r') order.
#include "c64_exact.cuh"
#include "internal.h"
#include "tile.cuh"

namespace sv {

// vbits > 0: the term index is packed below the sort key (sk = s << vbits |
// i) and no index array is written.
__global__ void __launch_bounds__(256) k_gate_keys(const uint64_t* __restrict__ keys, uint64_t n,
                                                   const BitPerm* __restrict__ perm,
                                                   uint64_t* __restrict__ sk, uint32_t* __restrict__ sidx,
                                                   uint32_t* __restrict__ hist, int passes, int vbits) {
  __shared__ uint32_t sh[MAX_PASSES][RADIX];
  __shared__ uint64_t fwd[16][16];
  for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) (&sh[0][0])[i] = 0;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) (&fwd[0][0])[i] = (&perm->fwd[0][0])[i];
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = permute_bits(fwd, keys[i]);
    if (vbits) {
      sk[i] = (s << vbits) | i;
    } else {
      sk[i] = s;
      sidx[i] = (uint32_t)i;
    }
    for (int p = 0; p < passes; ++p) atomicAdd(&sh[p][(s >> (RADIX_BITS * p)) & (RADIX - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) {
    uint32_t c = (&sh[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
}

void launch_gate_keys(const uint64_t* keys, uint64_t n, const GateParams& gp, uint64_t* sk,
                      uint32_t* sidx, uint32_t* hist, int passes, cudaStream_t st) {
  cudaMemsetAsync(hist, 0, sizeof(uint32_t) * MAX_PASSES * RADIX, st);
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_gate_keys<<<(unsigned)blocks, 256, 0, st>>>(keys, n, gp.perm, sk, sidx, hist, passes, gp.vbits);
}

// ------------------------------------------------------------------ heads
constexpr int HEAD_BLOCK = 256, HEAD_ITEMS = 16;

__global__ void __launch_bounds__(HEAD_BLOCK) k_group_heads(const uint64_t* __restrict__ sk, uint64_t n,
                                                            int shift, uint32_t* __restrict__ heads,
                                                            uint64_t* lookback, Ctl* ctl) {
  typedef TileLayout<HEAD_BLOCK, HEAD_ITEMS> L;
  __shared__ CompactShared<HEAD_BLOCK> cs;
  __shared__ uint64_t s_tile;
  const uint64_t tiles = (n + L::TILE - 1) / L::TILE;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd((unsigned long long*)&ctl->tile_counter[0], 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= tiles) break;
    const uint64_t base = tile * L::TILE;
    bool flag[HEAD_ITEMS];
    uint32_t pos[HEAD_ITEMS];
#pragma unroll
    for (int j = 0; j < HEAD_ITEMS; ++j) {
      uint64_t i = L::index(base, j);
      bool f = false;
      if (i < n) f = (i == 0) || ((sk[i] >> shift) != (sk[i - 1] >> shift));
      flag[j] = f;
    }
    tile_compact<HEAD_BLOCK, HEAD_ITEMS>(flag, pos, cs, lookback, tile, &ctl->err);
#pragma unroll
    for (int j = 0; j < HEAD_ITEMS; ++j)
      if (flag[j]) heads[cs.tile_base_out + pos[j]] = (uint32_t)L::index(base, j);
    if (tile == tiles - 1 && threadIdx.x == 0) ctl->count[0] = cs.tile_base_out + cs.tile_total;
    __syncthreads();
  }
}

// shift: sort-key bits below the group key (m, plus the packed index bits)
void launch_group_heads(const uint64_t* sk, uint64_t n, int shift, uint32_t* heads, uint64_t* lookback,
                        Ctl* ctl, cudaStream_t st) {
  uint64_t tiles = (n + HEAD_BLOCK * HEAD_ITEMS - 1) / (HEAD_BLOCK * HEAD_ITEMS);
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * (tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[0], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[0], 0, sizeof(uint64_t), st);
  if (n == 0) return;
  uint64_t grid = tiles < 148 * 4 ? tiles : 148 * 4;
  k_group_heads<<<(unsigned)grid, HEAD_BLOCK, 0, st>>>(sk, n, shift, heads, lookback, ctl);
}

// ------------------------------------------------------------------ apply
template <typename Real>
struct Cplx;
template <>
struct Cplx<double> {
  typedef double2 T;
};
template <>
struct Cplx<float> {
  typedef float2 T;
};

__device__ __forceinline__ double fma_r(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_r(float a, float b, float c) { return __fmaf_rn(a, b, c); }


constexpr int APPLY_TILE = 1024;                      // output slots per staged tile (multiple of 16)
constexpr int APPLY_ITEMS = APPLY_TILE / APPLY_BLOCK;  // 4

template <typename Real>
struct ApplySmem {
  typedef typename Cplx<Real>::T C2;
  C2 x[APPLY_TILE];                     // gathered member amplitudes
  C2 y[APPLY_TILE];                     // outputs, by slot
  uint64_t rest[APPLY_TILE / 2];        // squeezed key of each group
  uint32_t head[APPLY_TILE / 2 + 1];    // member offsets of the tile's groups
  uint16_t order[APPLY_TILE / 2];       // groups sorted by member count
  uint32_t present[APPLY_TILE / 2];     // member mask of each group
  uint8_t r[APPLY_TILE];                // member local index
  uint32_t size_count[17];
};

// One tile = APPLY_TILE consecutive output slots (group g, output r'), i.e.
// APPLY_TILE / 2^m whole groups.  Phase 1 stages the groups' members (local
// index and gathered amplitude) in shared memory with independent loads and
// orders the groups by member count, so that the lanes of a warp run
// multiply-add chains of equal length.  Phase 2 computes one output per slot
// in that order and parks it in shared memory under its original slot.
// Phase 3 drops exact zeros and writes the survivors in slot order.
template <typename Real>
__global__ void __launch_bounds__(APPLY_BLOCK, 4) k_gate_apply_staged(
    const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sidx, uint64_t n,
    const uint32_t* __restrict__ heads, const typename Cplx<Real>::T* __restrict__ amps_in,
    const GateParams gp, uint64_t* __restrict__ keys_out, typename Cplx<Real>::T* __restrict__ amps_out,
    uint64_t* __restrict__ probs_out, uint64_t* lookback, Ctl* ctl) {
  typedef TileLayout<APPLY_BLOCK, APPLY_ITEMS> L;
  typedef typename Cplx<Real>::T C2;
  extern __shared__ __align__(16) uint8_t s_dyn[];
  ApplySmem<Real>& sm = *reinterpret_cast<ApplySmem<Real>*>(s_dyn);
  __shared__ Real sU[512];
  __shared__ uint32_t s_re_nz[16], s_im_nz[16];
  __shared__ uint64_t s_inv[16][16];
  __shared__ CompactShared<APPLY_BLOCK> cs;
  __shared__ uint64_t s_tile;
  const int m = gp.m, d = 1 << m;
  for (int i = threadIdx.x; i < 2 * d * d; i += APPLY_BLOCK) sU[i] = (Real)gp.U[i];
  for (int i = threadIdx.x; i < 256; i += APPLY_BLOCK) (&s_inv[0][0])[i] = (&gp.perm->inv[0][0])[i];
  if (threadIdx.x < 16) {
    s_re_nz[threadIdx.x] = gp.re_nz[threadIdx.x];
    s_im_nz[threadIdx.x] = gp.im_nz[threadIdx.x];
  }
  const uint64_t G = ctl->count[0];
  const uint64_t S = G << m;
  const uint64_t tiles = (S + APPLY_TILE - 1) / APPLY_TILE;
  const uint32_t dmask = (uint32_t)d - 1u;
  const uint32_t groups_per_tile = (uint32_t)APPLY_TILE >> m;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd((unsigned long long*)&ctl->tile_counter[1], 1ull);
    if (threadIdx.x < 17) sm.size_count[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= tiles) break;
    const uint64_t base = tile * APPLY_TILE;
    // ---- phase 1: stage members, group heads and sizes
    const uint64_t g0 = base >> m;
    const uint64_t g1 = g0 + groups_per_tile < G ? g0 + groups_per_tile : G;
    const uint32_t ng = (uint32_t)(g1 - g0);
    const uint64_t mbase = heads[g0];
    const uint64_t mend = g1 < G ? (uint64_t)heads[g1] : n;
    uint32_t nm = (uint32_t)(mend - mbase);
    if (nm > APPLY_TILE) {  // only possible with duplicate keys: refuse instead of overrunning
      if (threadIdx.x == 0) atomicOr(&ctl->err, ERR_INVARIANT);
      nm = APPLY_TILE;
    }
    const int vb = gp.vbits;
    for (uint32_t k = threadIdx.x; k < ng; k += APPLY_BLOCK) {
      uint64_t h = heads[g0 + k];
      sm.head[k] = min((uint32_t)(h - mbase), nm);
      sm.rest[k] = sk[h] >> (m + vb);
    }
    if (threadIdx.x == 0) sm.head[ng] = nm;
    for (uint32_t k = threadIdx.x; k < nm; k += APPLY_BLOCK) {
      const uint64_t i = mbase + k;
      const uint64_t v = sk[i];
      sm.r[k] = (uint8_t)((v >> vb) & dmask);
      sm.x[k] = amps_in[vb ? (uint32_t)(v & ((1ull << vb) - 1ull)) : sidx[i]];
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < ng; k += APPLY_BLOCK) {
      uint32_t pm = 0;
      for (uint32_t q = sm.head[k]; q < sm.head[k + 1]; ++q) pm |= 1u << sm.r[q];
      sm.present[k] = pm;
      atomicAdd(&sm.size_count[__popc(pm)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // exclusive offsets of the size classes
      uint32_t acc = 0;
      for (int c = 0; c <= 16; ++c) {
        uint32_t v = sm.size_count[c];
        sm.size_count[c] = acc;
        acc += v;
      }
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < ng; k += APPLY_BLOCK)
      sm.order[atomicAdd(&sm.size_count[__popc(sm.present[k])], 1u)] = (uint16_t)k;
    __syncthreads();
    // ---- phase 2: one output per slot, groups in size order
    const uint32_t nslots = ng << m;
#pragma unroll
    for (int j = 0; j < APPLY_ITEMS; ++j) {
      const uint32_t ls = (uint32_t)j * APPLY_BLOCK + threadIdx.x;
      if (ls < nslots) {
        const uint32_t gl = sm.order[ls >> m];
        const uint32_t ro = ls & dmask;
        const uint32_t h = sm.head[gl];
        const uint32_t present = sm.present[gl];
        const uint32_t rnz = s_re_nz[ro] & present, inz = s_im_nz[ro] & present;
        uint32_t cols = rnz | inz;
        Real re = (Real)0, im = (Real)0;
        while (cols) {
          const int r = __ffs(cols) - 1;
          cols &= cols - 1u;
          const C2 x = sm.x[h + __popc(present & ((1u << r) - 1u))];
          const Real ur = sU[2 * (ro * d + r)], ui = sU[2 * (ro * d + r) + 1];
          if ((rnz >> r) & 1u) {
            re = fma_r(ur, x.x, re);
            im = fma_r(ur, x.y, im);
          }
          if ((inz >> r) & 1u) {
            re = fma_r(-ui, x.y, re);
            im = fma_r(ui, x.x, im);
          }
        }
        C2 yv;
        yv.x = re;
        yv.y = im;
        sm.y[(gl << m) | ro] = yv;
      }
    }
    __syncthreads();
    // ---- phase 3: drop zeros, write in slot order
    bool flag[APPLY_ITEMS];
    uint32_t pos[APPLY_ITEMS];
#pragma unroll
    for (int j = 0; j < APPLY_ITEMS; ++j) {
      const uint64_t slot = L::index(base, j);
      const uint32_t ls = (uint32_t)(slot - base);
      bool f = false;
      if (slot < S) {
        const C2 yv = sm.y[ls];
        f = !(yv.x == (Real)0 && yv.y == (Real)0);
      }
      flag[j] = f;
    }
    tile_compact<APPLY_BLOCK, APPLY_ITEMS>(flag, pos, cs, lookback, tile, &ctl->err);
#pragma unroll
    for (int j = 0; j < APPLY_ITEMS; ++j) {
      if (flag[j]) {
        const uint64_t slot = L::index(base, j);
        const uint32_t ls = (uint32_t)(slot - base);
        const uint32_t gl = ls >> m, ro = ls & dmask;
        const uint64_t key = permute_bits(s_inv, (sm.rest[gl] << m) | ro);
        const C2 yv = sm.y[ls];
        const uint64_t o = cs.tile_base_out + pos[j];
        keys_out[o] = key;
        amps_out[o] = yv;
        probs_out[o] = amp_prob_bits(yv);
      }
    }
    if (tile == tiles - 1 && threadIdx.x == 0) ctl->count[1] = cs.tile_base_out + cs.tile_total;
    __syncthreads();
  }
}

// One thread per partner group, GPT consecutive groups per thread (the
// loads of the GPT groups issued together: heads, first member's sort key,
// index, amplitude and key).  All 2^m outputs of a group are computed in
// registers with the fused multiply-add chain of Eq. (3) (present inputs in
// ascending r, products with a zero U component skipped); an output's key is
// the head member's key with the gate bits replaced by r'.  Nonzero outputs
// are placed in (group, r') order by a block scan and a decoupled look-back
// over tiles.
template <int MAXD>
__device__ __forceinline__ uint64_t deposit_r(uint32_t r, const int* q, int m) {
  uint64_t x = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (t < m) x |= (uint64_t)((r >> t) & 1u) << q[t];
  return x;
}

template <typename Real, int MAXD, int GPT>
__global__ void __launch_bounds__(APPLY_BLOCK) k_gate_apply(
    const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sidx, uint64_t n,
    const uint32_t* __restrict__ heads, const typename Cplx<Real>::T* __restrict__ amps_in,
    const uint64_t* __restrict__ keys_in, const GateParams gp, uint64_t* __restrict__ keys_out,
    typename Cplx<Real>::T* __restrict__ amps_out, uint64_t* __restrict__ probs_out, uint64_t* lookback,
    uint64_t max_tiles, Ctl* ctl) {
  typedef typename Cplx<Real>::T C2;
  constexpr int TILE_G = APPLY_BLOCK * GPT;
  constexpr int WARPS = APPLY_BLOCK / 32;
  __shared__ Real sU[2 * MAXD * MAXD];
  __shared__ uint32_t s_re_nz[MAXD], s_im_nz[MAXD];
  __shared__ uint32_t s_warp[WARPS];
  __shared__ uint64_t s_base;
  __shared__ uint32_t s_total;
  __shared__ uint64_t s_tile;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = gp.m, d = 1 << m;
  for (int i = tid; i < 2 * d * d; i += APPLY_BLOCK) sU[i] = (Real)gp.U[i];
  if (tid < d) {
    s_re_nz[tid] = gp.re_nz[tid];
    s_im_nz[tid] = gp.im_nz[tid];
  }
  int q[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) q[t] = gp.q[t];
  const uint64_t qmask = gp.qmask;
  const int vb = gp.vbits;
  const uint64_t imask = vb ? ((1ull << vb) - 1ull) : 0ull;
  const uint64_t G = ctl->count[0];
  const uint64_t tiles = (G + TILE_G - 1) / TILE_G;
  if (tiles > max_tiles) {  // the look-back buffer was sized for fewer tiles
    if (blockIdx.x == 0 && tid == 0) atomicOr(&ctl->err, ERR_INVARIANT);
    return;
  }
  __syncthreads();
  while (true) {
    if (tid == 0) s_tile = atomicAdd((unsigned long long*)&ctl->tile_counter[1], 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= tiles) break;
    const uint64_t g0 = tile * TILE_G + (uint64_t)tid * GPT;
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
      const uint32_t ix = ok ? (vb ? (uint32_t)(s0v[j] & imask) : sidx[hb[j]]) : 0u;
      x0v[j] = ok ? amps_in[ix] : C2();
      k0v[j] = ok ? keys_in[ix] : 0ull;
    }
    Real yr[GPT][MAXD], yi[GPT][MAXD];
    uint32_t keep[GPT];
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < GPT; ++j) {
      keep[j] = 0;
#pragma unroll
      for (int ro = 0; ro < MAXD; ++ro) yr[j][ro] = yi[j][ro] = (Real)0;
      if (g0 + j >= G) continue;
      const uint64_t h = hb[j], e = hb[j + 1];
      for (uint64_t i = h; i < e; ++i) {
        const uint64_t v = i == h ? s0v[j] : sk[i];
        const uint32_t r = (uint32_t)((v >> vb) & (uint64_t)(d - 1));
        const C2 x = i == h ? x0v[j] : amps_in[vb ? (uint32_t)(v & imask) : sidx[i]];
#pragma unroll
        for (int ro = 0; ro < MAXD; ++ro) {
          if (ro >= d) break;
          const bool rnz = (s_re_nz[ro] >> r) & 1u, inz = (s_im_nz[ro] >> r) & 1u;
          if (rnz) {
            const Real ur = sU[2 * (ro * d + r)];
            yr[j][ro] = fma_r(ur, x.x, yr[j][ro]);
            yi[j][ro] = fma_r(ur, x.y, yi[j][ro]);
          }
          if (inz) {
            const Real ui = sU[2 * (ro * d + r) + 1];
            yr[j][ro] = fma_r(-ui, x.y, yr[j][ro]);
            yi[j][ro] = fma_r(ui, x.x, yi[j][ro]);
          }
        }
      }
#pragma unroll
      for (int ro = 0; ro < MAXD; ++ro)
        if (ro < d && !(yr[j][ro] == (Real)0 && yi[j][ro] == (Real)0)) keep[j] |= 1u << ro;
      cnt += __popc(keep[j]);
    }
    // block exclusive scan of the counts, then the tile's global base
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const uint32_t v = lane < WARPS ? s_warp[lane] : 0u;
      uint32_t w = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < WARPS) s_warp[lane] = w - v;
      const uint32_t total = __shfl_sync(0xffffffffu, w, 31);
      const uint64_t base = lookback_exclusive_warp(lookback, tile, total, &ctl->err);
      if (lane == 0) {
        s_total = total;
        s_base = base;
      }
    }
    __syncthreads();
    uint64_t o = s_base + s_warp[warp] + (x - cnt);
#pragma unroll
    for (int j = 0; j < GPT; ++j) {
      if (!keep[j]) continue;
      const uint64_t rest = k0v[j] & ~qmask;
#pragma unroll
      for (int ro = 0; ro < MAXD; ++ro) {
        if (!((keep[j] >> ro) & 1u)) continue;
        keys_out[o] = rest | deposit_r<MAXD>((uint32_t)ro, q, m);
        C2 y;
        y.x = yr[j][ro];
        y.y = yi[j][ro];
        amps_out[o] = y;
        probs_out[o] = amp_prob_bits(y);
        ++o;
      }
    }
    if (tile == tiles - 1 && tid == 0) ctl->count[1] = s_base + s_total;
    __syncthreads();
  }
}

__global__ void k_flag_error(Ctl* ctl, uint32_t bits) { atomicOr(&ctl->err, bits); }

// Look-back descriptors the mat-vec may need for n input terms: one group
// per thread (group-per-thread kernel) or APPLY_TILE output slots per tile
// (staged kernel), whichever tiling has more tiles.
uint64_t gate_apply_tiles(uint64_t n, int m) {
  const uint64_t a = n / APPLY_BLOCK + 2, b = ((n << m) + APPLY_TILE - 1) / APPLY_TILE + 2;
  return a > b ? a : b;
}

// max_tiles (at least gate_apply_tiles(n, m)) sizes the look-back buffer.
void launch_gate_apply(int prec, const uint64_t* sk, const uint32_t* sidx, uint64_t n,
                       const uint32_t* heads, const void* amps_in, const uint64_t* keys_in, const GateParams& gp,
                       uint64_t* keys_out, void* amps_out, uint64_t* probs_out, uint64_t* lookback,
                       Ctl* ctl, cudaStream_t st, uint64_t max_tiles) {
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * (max_tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[1], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[1], 0, sizeof(uint64_t), st);
  if (n == 0) return;
  const uint64_t grid = max_tiles < 148 * 4 ? (max_tiles ? max_tiles : 1) : 148 * 4;
  const uint64_t staged_tiles = ((n << gp.m) + APPLY_TILE - 1) / APPLY_TILE;
  if (max_tiles < gate_apply_tiles(n, gp.m)) {  // the caller sized the look-back buffer too small
    k_flag_error<<<1, 1, 0, st>>>(ctl, ERR_INVARIANT);
    return;
  }
#define SV_GATE_APPLY(R, C2, MAXD, GPT)                                                                   \
  k_gate_apply<R, MAXD, GPT><<<(unsigned)grid, APPLY_BLOCK, 0, st>>>(sk, sidx, n, heads, (const C2*)amps_in, \
                                                                     keys_in, gp, keys_out, (C2*)amps_out,    \
                                                                     probs_out, lookback, max_tiles, ctl)
  if (prec == 0) {
    // complex128 is bound by the FP64 pipe: the staged kernel, whose warps run
    // groups of equal member count, keeps it busier than one group per thread
    static bool attr_set = false;
    if (!attr_set) {
      cudaFuncSetAttribute(k_gate_apply_staged<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(ApplySmem<double>));
      attr_set = true;
    }
    const uint64_t sgrid = staged_tiles < 148 * 4 ? (staged_tiles ? staged_tiles : 1) : 148 * 4;
    k_gate_apply_staged<double><<<(unsigned)sgrid, APPLY_BLOCK, sizeof(ApplySmem<double>), st>>>(
        sk, sidx, n, heads, (const double2*)amps_in, gp, keys_out, (double2*)amps_out, probs_out, lookback, ctl);
  } else {
    switch (gp.m) {
      case 1: SV_GATE_APPLY(float, float2, 2, 4); break;
      case 2: SV_GATE_APPLY(float, float2, 4, 2); break;
      case 3: SV_GATE_APPLY(float, float2, 8, 1); break;
      default: SV_GATE_APPLY(float, float2, 16, 1); break;
    }
  }
#undef SV_GATE_APPLY
}

}  // namespace sv
