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
#include "tile.cuh"
#include "batch.h"

namespace sv {

// ---------------------------------------------------------------- keys
__global__ void __launch_bounds__(256) k_seg_keys(const uint64_t* __restrict__ keys,
                                                  const uint16_t* __restrict__ seg, uint64_t n,
                                                  const SegGate* __restrict__ gates, int shift,
                                                  uint64_t* __restrict__ sk, uint32_t* __restrict__ sidx,
                                                  uint32_t* __restrict__ hist, int passes) {
  __shared__ uint32_t sh[MAX_PASSES][RADIX];
  for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t sg = seg[i];
    uint64_t s;
    if (gates[sg].m < 0) {
      s = ~0ull;  // term of a removed segment: sorts last and is cut off
    } else {
      s = ((uint64_t)sg << shift) | permute_bits(gates[sg].perm.fwd, keys[i]);
    }
    sk[i] = s;
    sidx[i] = (uint32_t)i;
    for (int p = 0; p < passes; ++p) atomicAdd(&sh[p][(s >> (RADIX_BITS * p)) & (RADIX - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) {
    const uint32_t c = (&sh[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
}

void launch_seg_keys(const uint64_t* keys, const uint16_t* seg, uint64_t n, const SegGate* gates, int shift,
                     uint64_t* sk, uint32_t* sidx, uint32_t* hist, int passes, cudaStream_t st) {
  cudaMemsetAsync(hist, 0, sizeof(uint32_t) * MAX_PASSES * RADIX, st);
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_seg_keys<<<(unsigned)blocks, 256, 0, st>>>(keys, seg, n, gates, shift, sk, sidx, hist, passes);
}

// ---------------------------------------------------------------- heads
constexpr int SH_BLOCK = 256, SH_ITEMS = 16;

__device__ __forceinline__ uint64_t seg_group_key(uint64_t s, int shift, const SegGate* gates) {
  const uint32_t sg = (uint32_t)(s >> shift);
  return s >> gates[sg].m;  // the segment id stays in the top bits
}

__global__ void __launch_bounds__(SH_BLOCK) k_seg_heads(const uint64_t* __restrict__ sk, uint64_t n, int shift,
                                                        const SegGate* __restrict__ gates,
                                                        uint32_t* __restrict__ heads, uint64_t* lookback,
                                                        Ctl* ctl) {
  typedef TileLayout<SH_BLOCK, SH_ITEMS> L;
  __shared__ CompactShared<SH_BLOCK> cs;
  __shared__ uint64_t s_tile;
  const uint64_t tiles = (n + L::TILE - 1) / L::TILE;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd((unsigned long long*)&ctl->tile_counter[0], 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
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
            seg_group_key(a, shift, gates) != seg_group_key(sk[i - 1], shift, gates);
      }
      flag[j] = f;
    }
    tile_compact<SH_BLOCK, SH_ITEMS>(flag, pos, cs, lookback, tile, &ctl->err);
#pragma unroll
    for (int j = 0; j < SH_ITEMS; ++j)
      if (flag[j]) heads[cs.tile_base_out + pos[j]] = (uint32_t)L::index(base, j);
    if (tile == tiles - 1 && threadIdx.x == 0) ctl->count[0] = cs.tile_base_out + cs.tile_total;
    __syncthreads();
  }
}

void launch_seg_heads(const uint64_t* sk, uint64_t n, int shift, const SegGate* gates, uint32_t* heads,
                      uint64_t* lookback, Ctl* ctl, cudaStream_t st) {
  const uint64_t tiles = (n + SH_BLOCK * SH_ITEMS - 1) / (SH_BLOCK * SH_ITEMS);
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * (tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[0], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[0], 0, sizeof(uint64_t), st);
  if (n == 0) return;
  const uint64_t grid = tiles < 148 * 4 ? tiles : 148 * 4;
  k_seg_heads<<<(unsigned)grid, SH_BLOCK, 0, st>>>(sk, n, shift, gates, heads, lookback, ctl);
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

constexpr int SA_BLOCK = 256, SA_ITEMS = 4;

// One thread per output slot (group, r'); every group owns 2^mmax slots and
// uses the first 2^m of them (m of its segment).  U entries are rounded to
// the amplitude precision exactly as in the single-state path.
template <typename Real>
__global__ void __launch_bounds__(SA_BLOCK) k_seg_apply(
    const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sidx, uint64_t n,
    const uint32_t* __restrict__ heads, const typename SCplx<Real>::T* __restrict__ amps_in, int shift,
    int mmax, const SegGate* __restrict__ gates, uint64_t* __restrict__ keys_out,
    typename SCplx<Real>::T* __restrict__ amps_out, uint64_t* __restrict__ probs_out,
    uint16_t* __restrict__ seg_out, uint64_t* lookback, Ctl* ctl) {
  typedef TileLayout<SA_BLOCK, SA_ITEMS> L;
  typedef typename SCplx<Real>::T C2;
  __shared__ CompactShared<SA_BLOCK> cs;
  __shared__ uint64_t s_tile;
  const uint64_t G = ctl->count[0];
  const uint64_t S = G << mmax;
  const uint64_t tiles = (S + L::TILE - 1) / L::TILE;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd((unsigned long long*)&ctl->tile_counter[1], 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= tiles) break;
    const uint64_t base = tile * L::TILE;
    bool flag[SA_ITEMS];
    uint32_t pos[SA_ITEMS];
    Real yr[SA_ITEMS], yi[SA_ITEMS];
    uint64_t ykey[SA_ITEMS];
    uint16_t ysg[SA_ITEMS];
#pragma unroll
    for (int j = 0; j < SA_ITEMS; ++j) {
      const uint64_t slot = L::index(base, j);
      Real re = (Real)0, im = (Real)0;
      bool f = false;
      uint64_t key = 0;
      uint32_t sg = 0;
      if (slot < S) {
        const uint64_t g = slot >> mmax;
        const uint32_t ro = (uint32_t)(slot & ((1u << mmax) - 1u));
        const uint64_t h = heads[g];
        const uint64_t e = g + 1 < G ? (uint64_t)heads[g + 1] : n;
        const uint64_t s0 = sk[h];
        sg = (uint32_t)(s0 >> shift);
        const SegGate& gt = gates[sg];
        const int m = gt.m;
        const int d = 1 << m;
        if ((int)ro < d) {
          uint32_t present = 0;
          for (uint64_t i = h; i < e; ++i) present |= 1u << (uint32_t)(sk[i] & (uint64_t)(d - 1));
          const uint32_t rnz = gt.re_nz[ro] & present, inz = gt.im_nz[ro] & present;
          uint32_t cols = rnz | inz;
          while (cols) {
            const int r = __ffs(cols) - 1;
            cols &= cols - 1u;
            const C2 x = amps_in[sidx[h + __popc(present & ((1u << r) - 1u))]];
            const Real ur = (Real)gt.U[2 * (ro * d + r)], ui = (Real)gt.U[2 * (ro * d + r) + 1];
            if ((rnz >> r) & 1u) {
              re = sfma(ur, x.x, re);
              im = sfma(ur, x.y, im);
            }
            if ((inz >> r) & 1u) {
              re = sfma(-ui, x.y, re);
              im = sfma(ui, x.x, im);
            }
          }
          const uint64_t local = s0 & ((1ull << shift) - 1ull);
          key = permute_bits(gt.perm.inv, ((local >> m) << m) | ro);
          f = !(re == (Real)0 && im == (Real)0);
        }
      }
      yr[j] = re;
      yi[j] = im;
      ykey[j] = key;
      ysg[j] = (uint16_t)sg;
      flag[j] = f;
    }
    tile_compact<SA_BLOCK, SA_ITEMS>(flag, pos, cs, lookback, tile, &ctl->err);
#pragma unroll
    for (int j = 0; j < SA_ITEMS; ++j) {
      if (flag[j]) {
        const uint64_t o = cs.tile_base_out + pos[j];
        keys_out[o] = ykey[j];
        C2 y;
        y.x = yr[j];
        y.y = yi[j];
        amps_out[o] = y;
        probs_out[o] = (uint64_t)__double_as_longlong(prob_of((double)yr[j], (double)yi[j]));
        seg_out[o] = ysg[j];
      }
    }
    if (tile == tiles - 1 && threadIdx.x == 0) ctl->count[1] = cs.tile_base_out + cs.tile_total;
    __syncthreads();
  }
}

void launch_seg_apply(int prec, const uint64_t* sk, const uint32_t* sidx, uint64_t n, const uint32_t* heads,
                      const void* amps_in, int shift, int mmax, const SegGate* gates, uint64_t* keys_out,
                      void* amps_out, uint64_t* probs_out, uint16_t* seg_out, uint64_t* lookback, Ctl* ctl,
                      uint64_t max_tiles, cudaStream_t st) {
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * (max_tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[1], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[1], 0, sizeof(uint64_t), st);
  if (n == 0) return;
  const uint64_t grid = max_tiles < 148 * 4 ? (max_tiles ? max_tiles : 1) : 148 * 4;
  if (prec == 0)
    k_seg_apply<double><<<(unsigned)grid, SA_BLOCK, 0, st>>>(sk, sidx, n, heads, (const double2*)amps_in, shift,
                                                             mmax, gates, keys_out, (double2*)amps_out,
                                                             probs_out, seg_out, lookback, ctl);
  else
    k_seg_apply<float><<<(unsigned)grid, SA_BLOCK, 0, st>>>(sk, sidx, n, heads, (const float2*)amps_in, shift,
                                                            mmax, gates, keys_out, (float2*)amps_out, probs_out,
                                                            seg_out, lookback, ctl);
}

// ---------------------------------------------------------------- segment bounds
// Segments are contiguous: record where each one starts and ends.
__global__ void k_seg_bounds(const uint16_t* __restrict__ seg, uint64_t n, uint64_t* __restrict__ start,
                             uint64_t* __restrict__ end) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint16_t s = seg[i];
    if (i == 0 || seg[i - 1] != s) start[s] = i;
    if (i + 1 == n || seg[i + 1] != s) end[s] = i + 1;
  }
}

void launch_seg_bounds(const uint16_t* seg, uint64_t n, uint64_t* start, uint64_t* end, int slots,
                       cudaStream_t st) {
  cudaMemsetAsync(start, 0, sizeof(uint64_t) * slots, st);
  cudaMemsetAsync(end, 0, sizeof(uint64_t) * slots, st);
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_seg_bounds<<<(unsigned)blocks, 256, 0, st>>>(seg, n, start, end);
}

// ---------------------------------------------------------------- segmented select
// The single-state radix select run for every segment at once: each segment
// has its own select state (prefix, target rank, counts and masses before
// its bin); a histogram level walks the terms in chunks, keeping the
// histogram of the segment it is in and flushing it when the segment changes.
constexpr int SS_BINS = SEL_BINS;

__device__ __forceinline__ void seg_add_u128(uint64_t* hi, uint64_t* lo, u128 v) {
  const uint64_t vl = (uint64_t)v;
  uint64_t vh = (uint64_t)(v >> 64);
  if (vl) {
    const uint64_t old = atomicAdd((unsigned long long*)lo, (unsigned long long)vl);
    if (old + vl < old) vh += 1;
  }
  if (vh) atomicAdd((unsigned long long*)hi, (unsigned long long)vh);
}

__device__ __forceinline__ bool seg_z_match(uint64_t hi, uint64_t lo, uint64_t ph, uint64_t pl, int bits) {
  if (bits <= 64) return ((hi ^ ph) >> (64 - bits)) == 0;
  if (hi != ph) return false;
  return ((lo ^ pl) >> (128 - bits)) == 0;
}

__device__ __forceinline__ void seg_digit(int bits, int* D, int* shift) {
  const int d = 128 - bits;
  *D = d < SEL_BITS ? d : SEL_BITS;
  *shift = 128 - bits - *D;
}

constexpr int SS_CHUNK = 16384;

__global__ void __launch_bounds__(256) k_segsel_hist(const uint64_t* __restrict__ probs,
                                                     const uint64_t* __restrict__ keys,
                                                     const uint16_t* __restrict__ seg, uint64_t n,
                                                     const SegSel* __restrict__ sel, uint32_t* __restrict__ g_cnt,
                                                     uint64_t* __restrict__ g_mass, uint32_t* err) {
  __shared__ uint32_t s_cnt[SS_BINS];
  __shared__ uint64_t s_mass[2 * SS_BINS];
  __shared__ uint32_t s_seg;
  const uint64_t chunks = (n + SS_CHUNK - 1) / SS_CHUNK;
  for (uint64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
    const uint64_t c0 = c * SS_CHUNK, c1 = c0 + SS_CHUNK < n ? c0 + SS_CHUNK : n;
    uint64_t i0 = c0;
    while (i0 < c1) {
      // the run of this chunk that belongs to one segment
      if (threadIdx.x == 0) s_seg = seg[i0];
      for (int b = threadIdx.x; b < SS_BINS; b += blockDim.x) {
        s_cnt[b] = 0;
        s_mass[2 * b] = s_mass[2 * b + 1] = 0;
      }
      __syncthreads();
      const uint32_t sg = s_seg;
      const SegSel& st = sel[sg];
      const bool active = st.active && !st.done;
      const int bits = (int)st.bits;
      int D, sh;
      seg_digit(bits, &D, &sh);
      uint64_t i1 = i0;
      // find the end of the run (segments are contiguous)
      {
        uint64_t lo = i0, hi = c1;  // first index in [i0, c1) with another segment
        while (lo < hi) {
          const uint64_t mid = (lo + hi) / 2;
          if (seg[mid] == sg) lo = mid + 1;
          else hi = mid;
        }
        i1 = lo;
      }
      if (active) {
        for (uint64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
          const uint64_t pb = probs[i];
          const uint64_t hi = ~pb;
          if (bits <= 64 && ((hi ^ st.prefix_hi) >> (64 - bits)) != 0) continue;
          const uint64_t lo = (bits > 64 || sh < 64) ? keys[i] : 0ull;
          if (!seg_z_match(hi, lo, st.prefix_hi, st.prefix_lo, bits)) continue;
          const u128 z = make_u128(hi, lo);
          const uint32_t dg = (uint32_t)(z >> sh) & ((1u << D) - 1u);
          atomicAdd(&s_cnt[dg], 1u);
          seg_add_u128(&s_mass[2 * dg], &s_mass[2 * dg + 1], fx_from_bits(pb, err));
        }
      }
      __syncthreads();
      if (active) {
        uint32_t* gc = g_cnt + (uint64_t)sg * SS_BINS;
        uint64_t* gm = g_mass + (uint64_t)sg * 2 * SS_BINS;
        for (int b = threadIdx.x; b < (1 << D); b += blockDim.x) {
          if (s_cnt[b]) {
            atomicAdd(&gc[b], s_cnt[b]);
            seg_add_u128(&gm[2 * b], &gm[2 * b + 1], make_u128(s_mass[2 * b], s_mass[2 * b + 1]));
          }
        }
      }
      __syncthreads();
      i0 = i1;
    }
  }
}

// One block per segment: pick the bin of the cut (same rule as the
// single-state select) and update the segment's select state.
__global__ void __launch_bounds__(256) k_segsel_pick(SegSel* __restrict__ sel, const uint32_t* __restrict__ g_cnt,
                                                     const uint64_t* __restrict__ g_mass, uint32_t* err) {
  __shared__ uint64_t w_c[8];
  __shared__ u128 w_m[8];
  __shared__ uint32_t s_first;
  SegSel& st = sel[blockIdx.x];
  if (!st.active || st.done) return;
  const uint32_t* cnt = g_cnt + (uint64_t)blockIdx.x * SS_BINS;
  const uint64_t* mass = g_mass + (uint64_t)blockIdx.x * 2 * SS_BINS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bits = (int)st.bits;
  int D, shift;
  seg_digit(bits, &D, &shift);
  const int nbins = 1 << D;
  const int per = (nbins + 255) / 256;
  const int b0 = tid * per;
  uint64_t my_c = 0;
  u128 my_m = 0;
  for (int b = b0; b < b0 + per && b < nbins; ++b) {
    my_c += cnt[b];
    my_m += make_u128(mass[2 * b], mass[2 * b + 1]);
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
    w_c[warp] = xc;
    w_m[warp] = xm;
  }
  if (tid == 0) s_first = 0xffffffffu;
  __syncthreads();
  uint64_t base_c = 0;
  u128 base_m = 0, total = 0;
  for (int w = 0; w < 8; ++w) {
    if (w < warp) {
      base_c += w_c[w];
      base_m += w_m[w];
    }
    total += w_m[w];
  }
  const uint64_t excl_c = base_c + xc - my_c;
  const u128 excl_m = base_m + xm - my_m;
  if (bits == 1 && tid == 0) {  // first level: every term of the segment is in some bin
    st.total_mass_hi = (uint64_t)(total >> 64);
    st.total_mass_lo = (uint64_t)total;
  }
  const uint64_t target = st.target;
  const uint64_t before_c = st.before_count;
  const u128 before_m = make_u128(st.before_mass_hi, st.before_mass_lo);
  {
    uint64_t cc = before_c + excl_c;
    for (int b = b0; b < b0 + per && b < nbins; ++b) {
      const uint32_t c = cnt[b];
      cc += c;
      if (c > 0 && cc >= target) {
        atomicMin(&s_first, (uint32_t)b);
        break;
      }
    }
  }
  __syncthreads();
  const uint32_t first = s_first;
  if (first == 0xffffffffu) {
    if (tid == 0) st.done = 2;
    return;
  }
  if ((int)first >= b0 && (int)first < b0 + per) {
    uint64_t bc = before_c + excl_c;
    u128 bm = before_m + excl_m;
    for (int b = b0; b < (int)first; ++b) {
      bc += cnt[b];
      bm += make_u128(mass[2 * b], mass[2 * b + 1]);
    }
    u128 prefix = make_u128(st.prefix_hi, st.prefix_lo);
    prefix |= ((u128)first) << shift;
    const int nb = bits + D;
    st.prefix_hi = (uint64_t)(prefix >> 64);
    st.prefix_lo = (uint64_t)prefix;
    st.bits = (uint32_t)nb;
    st.before_count = bc;
    st.before_mass_hi = (uint64_t)(bm >> 64);
    st.before_mass_lo = (uint64_t)bm;
    st.bin_count = cnt[first];
    if (nb == 128) {
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

void launch_segsel_level(const uint64_t* probs, const uint64_t* keys, const uint16_t* seg, uint64_t n, SegSel* sel,
                         int slots, uint32_t* g_cnt, uint64_t* g_mass, uint32_t* err, cudaStream_t st) {
  cudaMemsetAsync(g_cnt, 0, sizeof(uint32_t) * SS_BINS * slots, st);
  cudaMemsetAsync(g_mass, 0, sizeof(uint64_t) * 2 * SS_BINS * slots, st);
  if (n > 0) {
    const uint64_t chunks = (n + SS_CHUNK - 1) / SS_CHUNK;
    const uint64_t grid = chunks < 148 * 4 ? chunks : 148 * 4;
    k_segsel_hist<<<(unsigned)grid, 256, 0, st>>>(probs, keys, seg, n, sel, g_cnt, g_mass, err);
  }
  k_segsel_pick<<<slots, 256, 0, st>>>(sel, g_cnt, g_mass, err);
}

// Finish: one block per unresolved segment walks the terms of its current
// bin (already few) level after level inside shared memory.
constexpr int SF_CAP = 4096;

__global__ void __launch_bounds__(256) k_segsel_finish(const uint64_t* __restrict__ probs,
                                                       const uint64_t* __restrict__ keys,
                                                       const uint64_t* __restrict__ seg_start,
                                                       const uint64_t* __restrict__ seg_end, SegSel* sel,
                                                       uint32_t* err) {
  extern __shared__ __align__(16) uint8_t s_dyn[];
  uint64_t* bhi = reinterpret_cast<uint64_t*>(s_dyn);
  uint64_t* blo = bhi + SF_CAP;
  __shared__ uint32_t s_n;
  __shared__ uint32_t s_cnt[SS_BINS];
  __shared__ uint64_t s_mass[2 * SS_BINS];
  __shared__ uint64_t w_c[8];
  __shared__ u128 w_m[8];
  __shared__ uint32_t s_first;
  __shared__ SegSel st;  // the segment's select state, updated here and written back once
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    st = sel[blockIdx.x];
    s_n = 0;
  }
  __syncthreads();
  if (!st.active || st.done || st.bin_count > SF_CAP) return;
  {
    const int bits = (int)st.bits;
    for (uint64_t i = seg_start[blockIdx.x] + tid; i < seg_end[blockIdx.x]; i += blockDim.x) {
      const uint64_t hi = ~probs[i];
      if (bits <= 64 && ((hi ^ st.prefix_hi) >> (64 - bits)) != 0) continue;
      const uint64_t lo = keys[i];
      if (!seg_z_match(hi, lo, st.prefix_hi, st.prefix_lo, bits)) continue;
      const uint32_t p = atomicAdd(&s_n, 1u);
      if (p < SF_CAP) {
        bhi[p] = hi;
        blo[p] = lo;
      }
    }
  }
  __syncthreads();
  const uint32_t nb = s_n < SF_CAP ? s_n : SF_CAP;
  for (int it = 0; it < 128; ++it) {
    __syncthreads();
    if (st.done) break;
    const int bits = (int)st.bits;
    int D, shift;
    seg_digit(bits, &D, &shift);
    for (int b = tid; b < SS_BINS; b += blockDim.x) {
      s_cnt[b] = 0;
      s_mass[2 * b] = s_mass[2 * b + 1] = 0;
    }
    if (tid == 0) s_first = 0xffffffffu;
    __syncthreads();
    for (uint32_t i = tid; i < nb; i += blockDim.x) {
      if (!seg_z_match(bhi[i], blo[i], st.prefix_hi, st.prefix_lo, bits)) continue;
      const uint32_t dg = (uint32_t)(make_u128(bhi[i], blo[i]) >> shift) & ((1u << D) - 1u);
      atomicAdd(&s_cnt[dg], 1u);
      seg_add_u128(&s_mass[2 * dg], &s_mass[2 * dg + 1], fx_from_bits(~bhi[i], err));
    }
    __syncthreads();
    const int nbins = 1 << D;
    const int per = (nbins + 255) / 256;
    const int b0 = tid * per;
    uint64_t my_c = 0;
    u128 my_m = 0;
    for (int b = b0; b < b0 + per && b < nbins; ++b) {
      my_c += s_cnt[b];
      my_m += make_u128(s_mass[2 * b], s_mass[2 * b + 1]);
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
      w_c[warp] = xc;
      w_m[warp] = xm;
    }
    __syncthreads();
    uint64_t base_c = 0;
    u128 base_m = 0;
    for (int w = 0; w < warp; ++w) {
      base_c += w_c[w];
      base_m += w_m[w];
    }
    const uint64_t excl_c = base_c + xc - my_c;
    const u128 excl_m = base_m + xm - my_m;
    const uint64_t before_c = st.before_count;
    const u128 before_m = make_u128(st.before_mass_hi, st.before_mass_lo);
    const uint64_t target = st.target;
    {
      uint64_t cc = before_c + excl_c;
      for (int b = b0; b < b0 + per && b < nbins; ++b) {
        const uint32_t c = s_cnt[b];
        cc += c;
        if (c > 0 && cc >= target) {
          atomicMin(&s_first, (uint32_t)b);
          break;
        }
      }
    }
    __syncthreads();
    const uint32_t first = s_first;
    if (first == 0xffffffffu) {
      if (tid == 0) st.done = 2;
      __syncthreads();
      break;
    }
    if ((int)first >= b0 && (int)first < b0 + per) {
      uint64_t bc = before_c + excl_c;
      u128 bm = before_m + excl_m;
      for (int b = b0; b < (int)first; ++b) {
        bc += s_cnt[b];
        bm += make_u128(s_mass[2 * b], s_mass[2 * b + 1]);
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
      st.bin_count = s_cnt[first];
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
  if (tid == 0) sel[blockIdx.x] = st;
}

void launch_segsel_finish(const uint64_t* probs, const uint64_t* keys, const uint64_t* seg_start,
                          const uint64_t* seg_end, SegSel* sel, int slots, uint32_t* err, cudaStream_t st) {
  static bool attr_set = false;
  const size_t smem = 2 * sizeof(uint64_t) * SF_CAP;
  if (!attr_set) {
    cudaFuncSetAttribute(k_segsel_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  k_segsel_finish<<<slots, 256, smem, st>>>(probs, keys, seg_start, seg_end, sel, err);
}

// Renormalisation scale of every segment that found a cut.
__global__ void k_segsel_scale(SegSel* sel, int slots) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= slots) return;
  SegSel& st = sel[s];
  if (st.active && st.done == 1) st.scale = __ddiv_rn(1.0, __dsqrt_rn(fx_to_double(make_u128(st.cut_mass_hi, st.cut_mass_lo))));
}

void launch_segsel_scale(SegSel* sel, int slots, cudaStream_t st) {
  k_segsel_scale<<<(slots + 127) / 128, 128, 0, st>>>(sel, slots);
}

// ---------------------------------------------------------------- compaction
constexpr int SC_BLOCK = 256, SC_ITEMS = 8;

template <typename C2>
__device__ __forceinline__ C2 seg_scale(C2 a, double s);
template <>
__device__ __forceinline__ double2 seg_scale<double2>(double2 a, double s) {
  return make_double2(__dmul_rn(a.x, s), __dmul_rn(a.y, s));
}
template <>
__device__ __forceinline__ float2 seg_scale<float2>(float2 a, double s) {
  return make_float2(__double2float_rn(__dmul_rn((double)a.x, s)), __double2float_rn(__dmul_rn((double)a.y, s)));
}

// Keep, in each segment with a cut, the terms not after its cut (scaled);
// other segments keep everything unchanged.
template <typename C2>
__global__ void __launch_bounds__(SC_BLOCK) k_seg_truncate(
    const uint64_t* __restrict__ keys, const C2* __restrict__ amps, const uint64_t* __restrict__ probs,
    const uint16_t* __restrict__ seg, uint64_t n, const SegSel* __restrict__ sel, uint64_t* __restrict__ keys_out,
    C2* __restrict__ amps_out, uint64_t* __restrict__ probs_out, uint16_t* __restrict__ seg_out,
    uint64_t* lookback, Ctl* ctl) {
  typedef TileLayout<SC_BLOCK, SC_ITEMS> L;
  __shared__ CompactShared<SC_BLOCK> cs;
  __shared__ uint64_t s_tile;
  const uint64_t tiles = (n + L::TILE - 1) / L::TILE;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd((unsigned long long*)&ctl->tile_counter[2], 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= tiles) break;
    const uint64_t base = tile * L::TILE;
    bool flag[SC_ITEMS];
    uint32_t pos[SC_ITEMS];
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
      const uint64_t i = L::index(base, j);
      bool f = false;
      if (i < n) {
        const SegSel& st = sel[seg[i]];
        if (st.active && st.done == 1) {
          const uint64_t pb = probs[i];
          f = pb > st.cut_pbits || (pb == st.cut_pbits && keys[i] <= st.cut_key);
        } else {
          f = true;
        }
      }
      flag[j] = f;
    }
    tile_compact<SC_BLOCK, SC_ITEMS>(flag, pos, cs, lookback, tile, &ctl->err);
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
      if (flag[j]) {
        const uint64_t i = L::index(base, j);
        const uint64_t o = cs.tile_base_out + pos[j];
        const uint16_t sg = seg[i];
        const SegSel& st = sel[sg];
        C2 a = amps[i];
        uint64_t pb = probs[i];
        if (st.active && st.done == 1) {
          a = seg_scale<C2>(a, st.scale);
          pb = (uint64_t)__double_as_longlong(prob_of((double)a.x, (double)a.y));
        }
        keys_out[o] = keys[i];
        amps_out[o] = a;
        probs_out[o] = pb;
        seg_out[o] = sg;
      }
    }
    if (tile == tiles - 1 && threadIdx.x == 0) ctl->count[2] = cs.tile_base_out + cs.tile_total;
    __syncthreads();
  }
}

void launch_seg_truncate(int prec, const uint64_t* keys, const void* amps, const uint64_t* probs, const uint16_t* seg,
                         uint64_t n, const SegSel* sel, uint64_t* keys_out, void* amps_out, uint64_t* probs_out,
                         uint16_t* seg_out, uint64_t* lookback, Ctl* ctl, cudaStream_t st) {
  const uint64_t tiles = (n + SC_BLOCK * SC_ITEMS - 1) / (SC_BLOCK * SC_ITEMS);
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * (tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[2], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[2], 0, sizeof(uint64_t), st);
  if (n == 0) return;
  const uint64_t grid = tiles < 148 * 8 ? tiles : 148 * 8;
  if (prec == 0)
    k_seg_truncate<double2><<<(unsigned)grid, SC_BLOCK, 0, st>>>(keys, (const double2*)amps, probs, seg, n, sel,
                                                                 keys_out, (double2*)amps_out, probs_out, seg_out,
                                                                 lookback, ctl);
  else
    k_seg_truncate<float2><<<(unsigned)grid, SC_BLOCK, 0, st>>>(keys, (const float2*)amps, probs, seg, n, sel,
                                                                keys_out, (float2*)amps_out, probs_out, seg_out,
                                                                lookback, ctl);
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
