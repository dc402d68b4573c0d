// Truncation (Sec. III, Sec. IV-B) and readout (Sec. V).
//
// The paper sorts the terms by decreasing probability and keeps a prefix.
// Only the cut point is needed, so this file finds it by radix select on the
// 128-bit canonical composite Z = (~prob_bits, key): ascending Z is
// "probability descending, key ascending" because the bit pattern of a
// non-negative double orders like the double.  Each level histograms the
// next 11 bits of Z over the terms that match the bits fixed so far, with a
// count and an exact fixed-point mass per bin; a one-block kernel then finds
// the bin holding the rank-K term (top-k) or the term where the cumulative
// mass first reaches p * total (p-mass) and fixes its bits.  Once the chosen
// bin is small its terms are gathered and the remaining levels run inside one
// block.  A final compaction keeps every term not after the cut and applies
// the renormalisation.
#include "internal.h"
#include "tile.cuh"

namespace sv {

__device__ __forceinline__ void atomic_add_u128(uint64_t* hi, uint64_t* lo, u128 v) {
  uint64_t vl = (uint64_t)v, vh = (uint64_t)(v >> 64);
  if (vl) {
    uint64_t old = atomicAdd((unsigned long long*)lo, (unsigned long long)vl);
    if (old + vl < old) vh += 1;
  }
  if (vh) atomicAdd((unsigned long long*)hi, (unsigned long long)vh);
}

__device__ __forceinline__ bool z_matches(uint64_t hi, uint64_t lo, uint64_t ph, uint64_t pl,
                                          int bits) {
  if (bits <= 64) return bits == 0 || ((hi ^ ph) >> (64 - bits)) == 0;
  if (hi != ph) return false;
  return ((lo ^ pl) >> (128 - bits)) == 0;
}

// ---------------------------------------------------------------- init
__global__ void k_select_init(Ctl* ctl, int mode, uint64_t count_target) {
  ctl->sel_prefix_hi = 1ull << 63;  // ~sign bit of a non-negative double
  ctl->sel_prefix_lo = 0;
  ctl->sel_bits = 1;
  ctl->sel_mode = (uint32_t)mode;
  ctl->sel_done = 0;
  ctl->sel_compact = 0;
  ctl->sel_target_hi = 0;
  ctl->sel_target_lo = count_target;
  ctl->sel_before_count = 0;
  ctl->sel_before_mass_hi = 0;
  ctl->sel_before_mass_lo = 0;
  ctl->sel_bin_count = 0;
  ctl->compact_n = 0;
}

void launch_select_init(Ctl* ctl, int mode, uint64_t count_target, cudaStream_t st) {
  k_select_init<<<1, 1, 0, st>>>(ctl, mode, count_target);
}

// ---------------------------------------------------------------- histogram
__device__ __forceinline__ void sel_digit(int bits, int* D, int* shift) {
  int d = 128 - bits;
  *D = d < SEL_BITS ? d : SEL_BITS;
  *shift = 128 - bits - *D;
}

__device__ __forceinline__ uint32_t z_digit(uint64_t hi, uint64_t lo, int shift, int D) {
  u128 z = make_u128(hi, lo);
  return (uint32_t)(z >> shift) & ((1u << D) - 1u);
}

__global__ void __launch_bounds__(256) k_select_hist(const uint64_t* __restrict__ probs,
                                                     const uint64_t* __restrict__ keys, uint64_t n,
                                                     Ctl* ctl, uint32_t* __restrict__ g_cnt,
                                                     uint64_t* __restrict__ g_mass) {
  __shared__ uint32_t s_cnt[SEL_BINS];
  __shared__ uint64_t s_mass[SEL_BINS][2];
  if (ctl->sel_done) return;
  const int bits = (int)ctl->sel_bits;
  const uint64_t ph = ctl->sel_prefix_hi, pl = ctl->sel_prefix_lo;
  int D, shift;
  sel_digit(bits, &D, &shift);
  const bool need_lo = bits > 64 || shift < 64;
  for (int i = threadIdx.x; i < SEL_BINS; i += blockDim.x) {
    s_cnt[i] = 0;
    s_mass[i][0] = s_mass[i][1] = 0;
  }
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t pb = probs[i];
    uint64_t hi = ~pb;
    if (bits <= 64 && bits > 0 && ((hi ^ ph) >> (64 - bits)) != 0) continue;
    uint64_t lo = need_lo ? keys[i] : 0ull;
    if (bits > 64 && !z_matches(hi, lo, ph, pl, bits)) continue;
    uint32_t dg = z_digit(hi, lo, shift, D);
    atomicAdd(&s_cnt[dg], 1u);
    atomic_add_u128(&s_mass[dg][0], &s_mass[dg][1], fx_from_bits(pb, &ctl->err));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (1 << D); i += blockDim.x) {
    if (s_cnt[i]) {
      atomicAdd(&g_cnt[i], s_cnt[i]);
      atomic_add_u128(&g_mass[2 * i], &g_mass[2 * i + 1], make_u128(s_mass[i][0], s_mass[i][1]));
    }
  }
}

void launch_select_hist(const uint64_t* probs, const uint64_t* keys, uint64_t n, Ctl* ctl,
                        const SelectScratch& ss, cudaStream_t st) {
  cudaMemsetAsync(ss.hist_count, 0, sizeof(uint32_t) * SEL_BINS, st);
  cudaMemsetAsync(ss.hist_mass, 0, sizeof(uint64_t) * 2 * SEL_BINS, st);
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 4) blocks = 148 * 4;
  k_select_hist<<<(unsigned)blocks, 256, 0, st>>>(probs, keys, n, ctl, ss.hist_count, ss.hist_mass);
}

// ---------------------------------------------------------------- pick
constexpr int PICK_THREADS = 256;

__device__ __forceinline__ u128 shfl_up_u128(u128 v, int o) {
  uint64_t hi = __shfl_up_sync(0xffffffffu, (unsigned long long)(v >> 64), o);
  uint64_t lo = __shfl_up_sync(0xffffffffu, (unsigned long long)(uint64_t)v, o);
  return make_u128(hi, lo);
}

// Block-wide choice of the bin holding the cut, over `nbins` bins (count and
// 128-bit mass each).  Updates the select state in ctl.  Called by all
// PICK_THREADS threads of one block.
__device__ void block_pick(const uint32_t* cnt, const uint64_t* mass /* [nbins][2] */, Ctl* ctl,
                           double p) {
  __shared__ uint64_t w_c[PICK_THREADS / 32];
  __shared__ u128 w_m[PICK_THREADS / 32];
  __shared__ uint32_t s_first;
  __shared__ u128 s_total;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bits = (int)ctl->sel_bits;
  int D, shift;
  sel_digit(bits, &D, &shift);
  const int nbins = 1 << D;
  const int per = (nbins + PICK_THREADS - 1) / PICK_THREADS;
  const int b0 = tid * per;
  uint64_t my_c = 0;
  u128 my_m = 0;
  for (int b = b0; b < b0 + per && b < nbins; ++b) {
    my_c += cnt[b];
    my_m += make_u128(mass[2 * b], mass[2 * b + 1]);
  }
  // inclusive warp scans
  uint64_t xc = my_c;
  u128 xm = my_m;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t yc = __shfl_up_sync(0xffffffffu, (unsigned long long)xc, o);
    u128 ym = shfl_up_u128(xm, o);
    if (lane >= o) {
      xc += yc;
      xm += ym;
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
  for (int w = 0; w < PICK_THREADS / 32; ++w) {
    if (w < warp) {
      base_c += w_c[w];
      base_m += w_m[w];
    }
    total += w_m[w];
  }
  const uint64_t excl_c = base_c + xc - my_c;
  const u128 excl_m = base_m + xm - my_m;
  if (bits == 1 && tid == 0) {
    // first level: every term is in some bin, so this is S_N
    ctl->total_mass_hi = (uint64_t)(total >> 64);
    ctl->total_mass_lo = (uint64_t)total;
    if (ctl->sel_mode == 0) {
      double T = __dmul_rn(p, fx_to_double(total));
      u128 t = fx_from_bits((uint64_t)__double_as_longlong(T), &ctl->err);
      ctl->sel_target_hi = (uint64_t)(t >> 64);
      ctl->sel_target_lo = (uint64_t)t;
    }
    s_total = total;
  }
  __syncthreads();
  const uint32_t mode = ctl->sel_mode;
  const u128 target = make_u128(ctl->sel_target_hi, ctl->sel_target_lo);
  const uint64_t before_c = ctl->sel_before_count;
  const u128 before_m = make_u128(ctl->sel_before_mass_hi, ctl->sel_before_mass_lo);
  {
    uint64_t cc = before_c + excl_c;
    u128 cm = before_m + excl_m;
    for (int b = b0; b < b0 + per && b < nbins; ++b) {
      uint32_t c = cnt[b];
      cc += c;
      cm += make_u128(mass[2 * b], mass[2 * b + 1]);
      bool hit = c > 0 && (mode == 1 ? (u128)cc >= target : cm >= target);
      if (hit) {
        atomicMin(&s_first, (uint32_t)b);
        break;
      }
    }
  }
  __syncthreads();
  const uint32_t first = s_first;
  if (first == 0xffffffffu) {
    if (tid == 0) ctl->sel_done = 2;  // the target is never reached: no cut
    __syncthreads();
    return;
  }
  if ((int)first >= b0 && (int)first < b0 + per) {
    uint64_t bc = before_c + excl_c;
    u128 bm = before_m + excl_m;
    for (int b = b0; b < (int)first; ++b) {
      bc += cnt[b];
      bm += make_u128(mass[2 * b], mass[2 * b + 1]);
    }
    u128 prefix = make_u128(ctl->sel_prefix_hi, ctl->sel_prefix_lo);
    prefix |= ((u128)first) << shift;
    const int nb = bits + D;
    ctl->sel_prefix_hi = (uint64_t)(prefix >> 64);
    ctl->sel_prefix_lo = (uint64_t)prefix;
    ctl->sel_bits = (uint32_t)nb;
    ctl->sel_before_count = bc;
    ctl->sel_before_mass_hi = (uint64_t)(bm >> 64);
    ctl->sel_before_mass_lo = (uint64_t)bm;
    ctl->sel_bin_count = cnt[first];
    if (nb == 128) {
      uint64_t pbits = ~(uint64_t)(prefix >> 64);
      u128 sc = bm + fx_from_bits(pbits, &ctl->err);
      ctl->cut_pbits = pbits;
      ctl->cut_key = (uint64_t)prefix;
      ctl->cut_count = bc + 1;
      ctl->cut_mass_hi = (uint64_t)(sc >> 64);
      ctl->cut_mass_lo = (uint64_t)sc;
      ctl->sel_done = 1;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(PICK_THREADS) k_select_pick(Ctl* ctl, const uint32_t* cnt,
                                                              const uint64_t* mass, double p) {
  if (ctl->sel_done) return;
  block_pick(cnt, mass, ctl, p);
}

void launch_select_pick(Ctl* ctl, const SelectScratch& ss, double p, cudaStream_t st) {
  k_select_pick<<<1, PICK_THREADS, 0, st>>>(ctl, ss.hist_count, ss.hist_mass, p);
}

// ---------------------------------------------------------------- gather + finish
__global__ void __launch_bounds__(256) k_select_compact(const uint64_t* __restrict__ probs,
                                                        const uint64_t* __restrict__ keys,
                                                        uint64_t n, Ctl* ctl,
                                                        uint64_t* __restrict__ buf) {
  if (ctl->sel_done) return;
  const int bits = (int)ctl->sel_bits;
  const uint64_t ph = ctl->sel_prefix_hi, pl = ctl->sel_prefix_lo;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t hi = ~probs[i];
    if (bits <= 64 && ((hi ^ ph) >> (64 - bits)) != 0) continue;
    uint64_t lo = keys[i];
    if (!z_matches(hi, lo, ph, pl, bits)) continue;
    uint64_t pos = atomicAdd((unsigned long long*)&ctl->compact_n, 1ull);
    if (pos < FINISH_CAP) {
      buf[2 * pos] = hi;
      buf[2 * pos + 1] = lo;
    }
  }
}

void launch_select_compact(const uint64_t* probs, const uint64_t* keys, uint64_t n, Ctl* ctl,
                           const SelectScratch& ss, cudaStream_t st) {
  cudaMemsetAsync(&ctl->compact_n, 0, sizeof(uint64_t), st);
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 4) blocks = 148 * 4;
  k_select_compact<<<(unsigned)blocks, 256, 0, st>>>(probs, keys, n, ctl, ss.buf);
}

__global__ void __launch_bounds__(PICK_THREADS) k_select_finish(Ctl* ctl, const uint64_t* buf,
                                                                double p) {
  __shared__ uint32_t s_cnt[SEL_BINS];
  __shared__ uint64_t s_mass[2 * SEL_BINS];
  uint64_t nb = ctl->compact_n;
  if (nb > FINISH_CAP) nb = FINISH_CAP;
  for (int it = 0; it < 128; ++it) {
    __syncthreads();
    if (ctl->sel_done) break;
    const int bits = (int)ctl->sel_bits;
    const uint64_t ph = ctl->sel_prefix_hi, pl = ctl->sel_prefix_lo;
    int D, shift;
    sel_digit(bits, &D, &shift);
    for (int i = threadIdx.x; i < SEL_BINS; i += blockDim.x) {
      s_cnt[i] = 0;
      s_mass[2 * i] = s_mass[2 * i + 1] = 0;
    }
    __syncthreads();
    for (uint64_t i = threadIdx.x; i < nb; i += blockDim.x) {
      uint64_t hi = buf[2 * i], lo = buf[2 * i + 1];
      if (!z_matches(hi, lo, ph, pl, bits)) continue;
      uint32_t dg = z_digit(hi, lo, shift, D);
      atomicAdd(&s_cnt[dg], 1u);
      atomic_add_u128(&s_mass[2 * dg], &s_mass[2 * dg + 1], fx_from_bits(~hi, &ctl->err));
    }
    __syncthreads();
    block_pick(s_cnt, s_mass, ctl, p);
  }
}

void launch_select_finish(Ctl* ctl, const SelectScratch& ss, double p, cudaStream_t st) {
  k_select_finish<<<1, PICK_THREADS, 0, st>>>(ctl, ss.buf, p);
}

// ---------------------------------------------------------------- compaction
__global__ void k_set_scale(Ctl* ctl) {
  double sc = fx_to_double(make_u128(ctl->cut_mass_hi, ctl->cut_mass_lo));
  ctl->scale = __ddiv_rn(1.0, __dsqrt_rn(sc));
}

void launch_set_scale(Ctl* ctl, cudaStream_t st) { k_set_scale<<<1, 1, 0, st>>>(ctl); }

constexpr int TC_BLOCK = 256, TC_ITEMS = 4;

template <typename C2>
__device__ __forceinline__ C2 scale_amp(C2 a, double s);
template <>
__device__ __forceinline__ double2 scale_amp<double2>(double2 a, double s) {
  return make_double2(__dmul_rn(a.x, s), __dmul_rn(a.y, s));
}
template <>
__device__ __forceinline__ float2 scale_amp<float2>(float2 a, double s) {
  return make_float2(__double2float_rn(__dmul_rn((double)a.x, s)),
                     __double2float_rn(__dmul_rn((double)a.y, s)));
}

template <typename C2>
__global__ void __launch_bounds__(TC_BLOCK) k_truncate_compact(
    const uint64_t* __restrict__ keys, const C2* __restrict__ amps, const uint64_t* __restrict__ probs,
    uint64_t n, uint64_t* __restrict__ keys_out, C2* __restrict__ amps_out,
    uint64_t* __restrict__ probs_out, uint64_t* lookback, Ctl* ctl) {
  typedef TileLayout<TC_BLOCK, TC_ITEMS> L;
  __shared__ CompactShared<TC_BLOCK> cs;
  __shared__ uint64_t s_tile;
  const uint64_t pc = ctl->cut_pbits, kc = ctl->cut_key;
  const double s = ctl->scale;
  const uint64_t tiles = (n + L::TILE - 1) / L::TILE;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd((unsigned long long*)&ctl->tile_counter[2], 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= tiles) break;
    const uint64_t base = tile * L::TILE;
    bool flag[TC_ITEMS];
    uint32_t pos[TC_ITEMS];
    uint64_t kk[TC_ITEMS];
#pragma unroll
    for (int j = 0; j < TC_ITEMS; ++j) {
      uint64_t i = L::index(base, j);
      bool f = false;
      uint64_t key = 0;
      if (i < n) {
        uint64_t pb = probs[i];
        if (pb > pc) {
          f = true;
          key = keys[i];
        } else if (pb == pc) {
          key = keys[i];
          f = key <= kc;
        }
      }
      flag[j] = f;
      kk[j] = key;
    }
    tile_compact<TC_BLOCK, TC_ITEMS>(flag, pos, cs, lookback, tile, &ctl->err);
#pragma unroll
    for (int j = 0; j < TC_ITEMS; ++j) {
      if (flag[j]) {
        uint64_t i = L::index(base, j);
        uint64_t o = cs.tile_base_out + pos[j];
        C2 a = scale_amp<C2>(amps[i], s);
        keys_out[o] = kk[j];
        amps_out[o] = a;
        probs_out[o] = (uint64_t)__double_as_longlong(prob_of((double)a.x, (double)a.y));
      }
    }
    if (tile == tiles - 1 && threadIdx.x == 0) ctl->count[2] = cs.tile_base_out + cs.tile_total;
    __syncthreads();
  }
}

void launch_truncate_compact(int prec, const uint64_t* keys, const void* amps, const uint64_t* probs,
                             uint64_t n, uint64_t* keys_out, void* amps_out, uint64_t* probs_out,
                             uint64_t* lookback, Ctl* ctl, cudaStream_t st) {
  uint64_t tiles = (n + TC_BLOCK * TC_ITEMS - 1) / (TC_BLOCK * TC_ITEMS);
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * (tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[2], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[2], 0, sizeof(uint64_t), st);
  if (n == 0) return;
  uint64_t grid = tiles < 148 * 4 ? tiles : 148 * 4;
  if (prec == 0)
    k_truncate_compact<double2><<<(unsigned)grid, TC_BLOCK, 0, st>>>(
        keys, (const double2*)amps, probs, n, keys_out, (double2*)amps_out, probs_out, lookback, ctl);
  else
    k_truncate_compact<float2><<<(unsigned)grid, TC_BLOCK, 0, st>>>(
        keys, (const float2*)amps, probs, n, keys_out, (float2*)amps_out, probs_out, lookback, ctl);
}

// ---------------------------------------------------------------- peak
__global__ void __launch_bounds__(256) k_peak_max(const uint64_t* __restrict__ probs, uint64_t n,
                                                  Ctl* ctl) {
  uint64_t best = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t pb = probs[i];
    best = pb > best ? pb : best;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t y = __shfl_down_sync(0xffffffffu, (unsigned long long)best, o);
    best = y > best ? y : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long*)&ctl->peak_z_hi, best);
}

__global__ void __launch_bounds__(256) k_peak_key(const uint64_t* __restrict__ probs,
                                                  const uint64_t* __restrict__ keys, uint64_t n,
                                                  Ctl* ctl) {
  const uint64_t pmax = ctl->peak_z_hi;
  uint64_t best = ~0ull;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    if (probs[i] == pmax) {
      uint64_t k = keys[i];
      best = k < best ? k : best;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t y = __shfl_down_sync(0xffffffffu, (unsigned long long)best, o);
    best = y < best ? y : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMin((unsigned long long*)&ctl->peak_z_lo, best);
}

void launch_peak(const uint64_t* probs, const uint64_t* keys, uint64_t n, Ctl* ctl, cudaStream_t st) {
  cudaMemsetAsync(&ctl->peak_z_hi, 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->peak_z_lo, 0xff, sizeof(uint64_t), st);
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_peak_max<<<(unsigned)blocks, 256, 0, st>>>(probs, n, ctl);
  k_peak_key<<<(unsigned)blocks, 256, 0, st>>>(probs, keys, n, ctl);
}

// ---------------------------------------------------------------- readout helpers
__global__ void k_iota(uint32_t* v, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    v[i] = (uint32_t)i;
}

void launch_iota(uint32_t* v, uint64_t n, cudaStream_t st) {
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_iota<<<(unsigned)blocks, 256, 0, st>>>(v, n);
}

__global__ void k_not_bits_gather(const uint64_t* __restrict__ probs, const uint32_t* __restrict__ idx,
                                  uint64_t n, uint64_t* __restrict__ out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = ~probs[idx[i]] & ~(1ull << 63);  // ~pbits without its constant top bit
}

void launch_not_bits_gather(const uint64_t* probs, const uint32_t* idx, uint64_t n, uint64_t* out,
                            cudaStream_t st) {
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_not_bits_gather<<<(unsigned)blocks, 256, 0, st>>>(probs, idx, n, out);
}

template <typename C2>
__global__ void k_gather_terms(const uint32_t* __restrict__ idx, uint64_t n,
                               const uint64_t* __restrict__ keys, const C2* __restrict__ amps,
                               const uint64_t* __restrict__ probs, uint64_t* __restrict__ keys_out,
                               double2* __restrict__ amps_out, uint64_t* __restrict__ probs_out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t j = idx[i];
    if (keys_out) keys_out[i] = keys[j];
    if (amps_out) {
      C2 a = amps[j];
      amps_out[i] = make_double2((double)a.x, (double)a.y);
    }
    if (probs_out) probs_out[i] = probs[j];
  }
}

void launch_gather_terms(int prec, const uint32_t* idx, uint64_t n, const uint64_t* keys,
                         const void* amps, const uint64_t* probs, uint64_t* keys_out,
                         double* amps_out, uint64_t* probs_out, cudaStream_t st) {
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  if (prec == 0)
    k_gather_terms<double2><<<(unsigned)blocks, 256, 0, st>>>(
        idx, n, keys, (const double2*)amps, probs, keys_out, (double2*)amps_out, probs_out);
  else
    k_gather_terms<float2><<<(unsigned)blocks, 256, 0, st>>>(
        idx, n, keys, (const float2*)amps, probs, keys_out, (double2*)amps_out, probs_out);
}

// ---------------------------------------------------------------- load
template <typename C2>
__device__ __forceinline__ C2 from_double2(double2 a);
template <>
__device__ __forceinline__ double2 from_double2<double2>(double2 a) {
  return a;
}
template <>
__device__ __forceinline__ float2 from_double2<float2>(double2 a) {
  return make_float2(__double2float_rn(a.x), __double2float_rn(a.y));
}

template <typename C2>
__global__ void __launch_bounds__(TC_BLOCK) k_load_compact(const uint64_t* __restrict__ skeys,
                                                           const uint32_t* __restrict__ idx, uint64_t n,
                                                           const double2* __restrict__ amps_in,
                                                           uint64_t* __restrict__ keys_out,
                                                           C2* __restrict__ amps_out,
                                                           uint64_t* __restrict__ probs_out,
                                                           uint64_t* lookback, Ctl* ctl) {
  typedef TileLayout<TC_BLOCK, TC_ITEMS> L;
  __shared__ CompactShared<TC_BLOCK> cs;
  __shared__ uint64_t s_tile;
  const uint64_t tiles = (n + L::TILE - 1) / L::TILE;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd((unsigned long long*)&ctl->tile_counter[2], 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= tiles) break;
    const uint64_t base = tile * L::TILE;
    bool flag[TC_ITEMS];
    uint32_t pos[TC_ITEMS];
    C2 av[TC_ITEMS];
#pragma unroll
    for (int j = 0; j < TC_ITEMS; ++j) {
      uint64_t i = L::index(base, j);
      bool f = false;
      if (i < n) {
        if (i > 0 && skeys[i] == skeys[i - 1])
          atomicAdd((unsigned long long*)&ctl->count[3], 1ull);
        C2 a = from_double2<C2>(amps_in[idx[i]]);
        av[j] = a;
        f = !(a.x == 0 && a.y == 0);
      }
      flag[j] = f;
    }
    tile_compact<TC_BLOCK, TC_ITEMS>(flag, pos, cs, lookback, tile, &ctl->err);
#pragma unroll
    for (int j = 0; j < TC_ITEMS; ++j) {
      if (flag[j]) {
        uint64_t i = L::index(base, j);
        uint64_t o = cs.tile_base_out + pos[j];
        keys_out[o] = skeys[i];
        amps_out[o] = av[j];
        probs_out[o] = (uint64_t)__double_as_longlong(prob_of((double)av[j].x, (double)av[j].y));
      }
    }
    if (tile == tiles - 1 && threadIdx.x == 0) ctl->count[2] = cs.tile_base_out + cs.tile_total;
    __syncthreads();
  }
}

void launch_load_compact(int prec, const uint64_t* sorted_keys, const uint32_t* idx, uint64_t n,
                         const double* amps_in, uint64_t* keys_out, void* amps_out,
                         uint64_t* probs_out, uint64_t* lookback, Ctl* ctl, cudaStream_t st) {
  uint64_t tiles = (n + TC_BLOCK * TC_ITEMS - 1) / (TC_BLOCK * TC_ITEMS);
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * (tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[2], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[2], 0, sizeof(uint64_t) * 2, st);
  if (n == 0) return;
  uint64_t grid = tiles < 148 * 4 ? tiles : 148 * 4;
  if (prec == 0)
    k_load_compact<double2><<<(unsigned)grid, TC_BLOCK, 0, st>>>(
        sorted_keys, idx, n, (const double2*)amps_in, keys_out, (double2*)amps_out, probs_out,
        lookback, ctl);
  else
    k_load_compact<float2><<<(unsigned)grid, TC_BLOCK, 0, st>>>(
        sorted_keys, idx, n, (const double2*)amps_in, keys_out, (float2*)amps_out, probs_out,
        lookback, ctl);
}

}  // namespace sv
