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
#include "launch.cuh"
#include "c64_exact.cuh"
#include "select.cuh"
#include "tile.cuh"

namespace sv {

// Natural key of a stored key (identity when the keys are natural).
__device__ __forceinline__ uint64_t natural_key(const uint64_t* nat, uint64_t k) {
  return nat ? to_natural(nat, k) : k;
}

// The list is the window buffer when the window pass set use_window, else
// all terms: the choice and the list length are read on the device, so the
// select can be enqueued before the window is known.  Block b scans a
// contiguous chunk of at least SH_CHUNK terms (each block flushes up to
// 3 * SEL_BINS global atomics, so blocks get a large share each).
constexpr int SH_UNROLL = 8;
constexpr uint64_t SH_CHUNK = 4096;
__global__ void __launch_bounds__(256, 4) k_select_hist(const uint64_t* __restrict__ probs,
                                                     const uint64_t* __restrict__ keys, uint64_t n,
                                                     const uint64_t* __restrict__ wp, const uint32_t* __restrict__ wi,
                                                     Ctl* ctl, uint32_t* __restrict__ g_cnt,
                                                     uint64_t* __restrict__ g_mass) {
  pdl_prologue();
  __shared__ uint32_t s_cnt[SEL_BINS];
  __shared__ uint64_t s_mass[2 * SEL_BINS];
  if (ctl->sel_done) return;
  if (ctl->sel_gated && ctl->sel_bin_count <= (uint64_t)FINISH_CAP) return;  // the finish takes over
  const bool win = ctl->use_window != 0;
  const uint64_t* P = win ? wp : probs;
  const uint64_t* nat = ctl->nat;
  const uint64_t nn = win ? ctl->win_n : n;
  uint64_t chunk = (nn + gridDim.x - 1) / gridDim.x;
  if (chunk < SH_CHUNK) chunk = SH_CHUNK;
  const uint64_t c0 = blockIdx.x * chunk;
  if (c0 >= nn) return;
  const uint64_t c1 = c0 + chunk < nn ? c0 + chunk : nn;
  const int bits = (int)ctl->sel_bits;
  const uint64_t ph = ctl->sel_prefix_hi, pl = ctl->sel_prefix_lo;
  int D, shift;
  sel_digit(bits, &D, &shift);
  const bool need_lo = bits > 64 || shift < 64;
  for (int i = threadIdx.x; i < SEL_BINS; i += blockDim.x) {
    s_cnt[i] = 0;
    s_mass[2 * i] = s_mass[2 * i + 1] = 0;
  }
  __syncthreads();
  BinCache cache;
  // SH_UNROLL terms per thread at a time, their loads issued together (the
  // bins' sums are exact integers, so the order of the additions is free)
  for (uint64_t i0 = c0 + threadIdx.x; i0 < c1; i0 += (uint64_t)SH_UNROLL * blockDim.x) {
    uint64_t pbv[SH_UNROLL], lov[SH_UNROLL];
#pragma unroll
    for (int u = 0; u < SH_UNROLL; ++u) {
      const uint64_t i = i0 + (uint64_t)u * blockDim.x;
      pbv[u] = i < c1 ? P[i] : 0ull;
    }
    if (need_lo) {  // the stored key (made natural) only where a tie on the probability needs it
#pragma unroll
      for (int u = 0; u < SH_UNROLL; ++u) {
        const uint64_t i = i0 + (uint64_t)u * blockDim.x;
        lov[u] = i < c1 ? keys[win ? (uint64_t)wi[i] : i] : 0ull;
      }
    }
#pragma unroll
    for (int u = 0; u < SH_UNROLL; ++u) {
      const uint64_t i = i0 + (uint64_t)u * blockDim.x;
      if (i >= c1) continue;
      const uint64_t pb = pbv[u];
      const uint64_t hi = ~pb;
      if (bits <= 64 && bits > 0 && ((hi ^ ph) >> (64 - bits)) != 0) continue;
      const uint64_t lo = need_lo ? natural_key(nat, lov[u]) : 0ull;
      if (bits > 64 && !z_matches(hi, lo, ph, pl, bits)) continue;
      hist_add(z_digit(hi, lo, shift, D), pb, s_cnt, s_mass, &ctl->err, cache);
    }
  }
  bin_cache_flush(cache, s_cnt, s_mass);
  __syncthreads();
  for (int i = threadIdx.x; i < (1 << D); i += blockDim.x) {
    if (s_cnt[i]) {
      atomicAdd(&g_cnt[i], s_cnt[i]);
      atomic_add_u128(&g_mass[2 * i], &g_mass[2 * i + 1], make_u128(s_mass[2 * i], s_mass[2 * i + 1]));
    }
  }
}

// The histogram arrives cleared: it is zero when allocated, and the pick that
// follows every histogram level clears it after reading it.
void launch_select_hist(const uint64_t* probs, const uint64_t* keys, uint64_t n, Ctl* ctl,
                        const SelectScratch& ss, cudaStream_t st) {
  if (n == 0) return;
  uint64_t blocks = (n + SH_CHUNK - 1) / SH_CHUNK;
  if (blocks > 148 * 4) blocks = 148 * 4;  // four resident per SM (40 KB of bins each)
  launch_pdl(k_select_hist, (unsigned)blocks, 256, 0, st, probs, keys, n, ss.win_p, ss.win_i, ctl, ss.hist_count,
             ss.hist_mass);
}

// ---------------------------------------------------------------- sample window
// The cut is located from a sample first: from SAMPLE_N probabilities at
// evenly spaced positions the sample rank of the cut is estimated (count:
// K * SAMPLE_N / N, two order statistics found by a radix select; mass: the
// prefix of the sorted sample whose mass fraction reaches p) and a window of +-4 binomial standard deviations (+16)
// around it is turned into a probability interval [lo, hi].  One streaming
// pass then sums the exact fixed-point mass of all terms, counts and sums the
// terms above hi, and gathers the terms inside [lo, hi].  If the window
// provably holds the cut, the radix select runs on the window only; else it
// runs on all terms.  The sample only steers the work: the cut found is the
// exact one either way.
constexpr int SAMPLE_N = 8192;
constexpr int SAMPLE_THREADS = 1024;

// LSD radix sort (4 passes of 8 bits) of SAMPLE_N 32-bit keys in shared
// memory by one 1024-thread block.  Warp w owns keys [w*256, (w+1)*256)
// lane-interleaved; ranks come from __match_any_sync and per-warp digit
// counters, so each pass is stable.  The result ends in `a`.
__device__ void block_sort_samples(uint32_t* a, uint32_t* tmp, uint32_t* whist /* [32][256] */,
                                   uint32_t* dsum /* [256] */, uint32_t* wtot /* [32] */) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  constexpr int ITEMS = SAMPLE_N / SAMPLE_THREADS;  // 8
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 8 * pass;
    uint32_t k[ITEMS], d[ITEMS], rk[ITEMS];
    for (int i = lane; i < 256; i += 32) whist[warp * 256 + i] = 0;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      k[i] = a[warp * 256 + i * 32 + lane];
      d[i] = (k[i] >> shift) & 255u;
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      uint32_t peers = __match_any_sync(0xffffffffu, d[i]);
      int leader = __ffs(peers) - 1;
      uint32_t old = 0;
      if (lane == leader) {
        old = whist[warp * 256 + d[i]];
        whist[warp * 256 + d[i]] = old + __popc(peers);
      }
      rk[i] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
      __syncwarp();
    }
    __syncthreads();
    uint32_t tot = 0;
    if (tid < 256) {
      for (int w = 0; w < 32; ++w) {
        uint32_t c = whist[w * 256 + tid];
        whist[w * 256 + tid] = tot;
        tot += c;
      }
    }
    // exclusive scan of the 256 digit totals
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wtot[warp] = x;
    __syncthreads();
    if (tid < 256) {
      uint32_t base = 0;
      for (int w = 0; w < warp; ++w) base += wtot[w];
      dsum[tid] = base + x - tot;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) tmp[dsum[d[i]] + whist[warp * 256 + d[i]] + rk[i]] = k[i];
    __syncthreads();
    uint32_t* t = a;
    a = tmp;
    tmp = t;
  }
}

// Values of ascending ranks r[0] and r[1] among the SAMPLE_N 32-bit keys in
// a (shared memory), by a radix select: four 8-bit digits, most significant
// first; for each rank a histogram of the digit among the keys that match the
// digits fixed so far (warp-aggregated shared atomics), then the bin that
// holds the rank.  out[t] receives the value of rank r[t].
__device__ void block_select_two(const uint32_t* a, const int* r, uint32_t* hist /* [2][256] */,
                                 uint32_t* pref /* [2] */, uint32_t* rem /* [2] */) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int ITEMS = SAMPLE_N / SAMPLE_THREADS;
  uint32_t k[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) k[i] = a[i * SAMPLE_THREADS + tid];
  if (tid < 2) {
    pref[tid] = 0;
    rem[tid] = (uint32_t)r[tid];
  }
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int i = tid; i < 512; i += SAMPLE_THREADS) hist[i] = 0;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const uint32_t pf = pref[t];
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const bool match = pass == 0 || ((k[i] ^ pf) >> (shift + 8)) == 0;
        const uint32_t d = match ? (k[i] >> shift) & 255u : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (d < 256u && lane == __ffs(peers) - 1) atomicAdd(&hist[t * 256 + d], (uint32_t)__popc(peers));
      }
    }
    __syncthreads();
    if (warp < 2) {  // warp t finds the bin of rank rem[t]: lane l scans bins 8l .. 8l + 7
      const uint32_t* h = hist + warp * 256;
      uint32_t c[8], sum = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        c[b] = h[lane * 8 + b];
        sum += c[b];
      }
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      const uint32_t before = x - sum, want = rem[warp];
      if (want >= before && want < x) {  // exactly one lane holds the rank
        uint32_t acc = before;
        for (int b = 0; b < 8; ++b) {
          if (want < acc + c[b]) {
            pref[warp] |= (uint32_t)(lane * 8 + b) << shift;
            rem[warp] = want - acc;
            break;
          }
          acc += c[b];
        }
      }
    }
    __syncthreads();
  }
}

// The cut is located from a sample first: SAMPLE_N probabilities at evenly
// spaced positions, reduced to the top 32 bits of their inverted bit pattern
// (exponent and 20 mantissa bits), are ranked in shared memory; the sample
// rank of the cut is estimated (count: K * SAMPLE_N / N, and only the two
// window ends are selected; mass: the sorted sample's prefix whose mass
// fraction reaches p) and a window of +-4 binomial
// standard deviations (+16; doubled for mass) around it becomes a
// probability interval [lo, hi], rounded outwards.  The sample only steers
// the work: the cut found afterwards is the exact one either way.
__global__ void __launch_bounds__(SAMPLE_THREADS) k_sample_window(const uint64_t* __restrict__ probs,
                                                                  uint64_t n, Ctl* ctl, int mode,
                                                                  uint64_t count_target, double p,
                                                                  bool total_known) {
  pdl_prologue();
  extern __shared__ __align__(16) uint8_t s_dyn[];
  uint32_t* a = reinterpret_cast<uint32_t*>(s_dyn);
  uint32_t* tmp = a + SAMPLE_N;
  uint32_t* whist = tmp + SAMPLE_N;
  double* pre = reinterpret_cast<double*>(whist + 32 * 256);
  __shared__ uint32_t dsum[256], wtot[32];
  __shared__ int s_rank;
  const int tid = threadIdx.x;
  if (tid < 8) (&ctl->win_n)[tid] = 0;  // win_n .. below_mass_lo, summed by the window pass
  if (tid == 8) ctl->pmax_bits = 0;     // the largest probability, taken by the window pass
  if (!total_known && tid == 0) ctl->total_mass_hi = ctl->total_mass_lo = 0;  // the pass sums the total too
  // stratified random sample: one term at a hashed offset inside each of
  // SAMPLE_N equal strata (a fixed stride would alias with the 2^m-periodic
  // layout of the candidates)
  {
    constexpr int SI = SAMPLE_N / SAMPLE_THREADS;
    uint64_t idx[SI], v[SI];
#pragma unroll
    for (int t = 0; t < SI; ++t) {
      const uint64_t j = (uint64_t)(tid + t * SAMPLE_THREADS);
      const uint64_t b0 = j * (n / SAMPLE_N) + (j * (n % SAMPLE_N)) / SAMPLE_N;
      const uint64_t b1 = (j + 1) * (n / SAMPLE_N) + ((j + 1) * (n % SAMPLE_N)) / SAMPLE_N;
      uint64_t h = j * 0x9E3779B97F4A7C15ull;
      h ^= h >> 31;
      h *= 0xBF58476D1CE4E5B9ull;
      h ^= h >> 29;
      idx[t] = b1 > b0 ? b0 + h % (b1 - b0) : (b0 < n ? b0 : n - 1);
    }
#pragma unroll
    for (int t = 0; t < SI; ++t) v[t] = probs[idx[t]];  // the probes in flight together
#pragma unroll
    for (int t = 0; t < SI; ++t)
      a[tid + t * SAMPLE_THREADS] = (uint32_t)((~v[t]) >> 31);  // drop the constant top bit, keep 32 bits
  }
  __syncthreads();
  if (mode == 1) {  // by count: only two order statistics of the sample are needed
    __shared__ int s_r[2];
    __shared__ uint32_t s_pref[2], s_rem[2];
    if (tid == 0) {
      const double rr = (double)count_target * SAMPLE_N / (double)n - 1.0;
      const int r = (int)(rr < 0 ? 0 : (rr > SAMPLE_N - 1 ? SAMPLE_N - 1 : rr));
      const double q = (r + 1.0) / SAMPLE_N;
      const int delta = (int)(4.0 * sqrt(SAMPLE_N * q * (1.0 - q)) + 16.0);
      s_r[0] = r - delta;
      s_r[1] = r + delta;
    }
    __syncthreads();
    const int rh = s_r[0], rl = s_r[1];
    const int rs[2] = {rh < 0 ? 0 : rh, rl > SAMPLE_N - 1 ? SAMPLE_N - 1 : rl};
    block_select_two(a, rs, whist, s_pref, s_rem);
    if (tid == 0) {
      // inverted patterns: a smaller value is a larger probability
      ctl->win_hi = rh <= 0 ? 0x7ff0000000000000ull : ~(((uint64_t)s_pref[0] << 31) | (1ull << 63));
      ctl->win_lo = rl >= SAMPLE_N - 1 ? 0ull : ~((((uint64_t)s_pref[1] << 31) | (1ull << 63)) | 0x7fffffffull);
    }
    return;
  }
  block_sort_samples(a, tmp, whist, dsum, wtot);  // 4 passes: result back in a
  {
    // the sample rank where the sorted sample's mass first reaches p of its
    // total: a block-wide scan of the threads' 8-value sums, then the one
    // thread whose range holds the crossing walks its values (a steering
    // estimate in double; the exact cut is found afterwards)
    constexpr int PER = SAMPLE_N / SAMPLE_THREADS;
    const int lane = tid & 31, warp = tid >> 5;
    double v[PER], loc = 0.0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      v[k] = __longlong_as_double((long long)~(((uint64_t)a[tid * PER + k] << 31) | (1ull << 63)));
      loc += v[k];
    }
    double x = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) pre[warp] = x;
    if (tid == 0) s_rank = SAMPLE_N - 1;
    __syncthreads();
    if (warp == 0) {
      double w = pre[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      pre[32 + lane] = w;  // inclusive over the warps
    }
    __syncthreads();
    const double total = pre[32 + 31];
    const double goal = p * total;
    double acc = (warp > 0 ? pre[32 + warp - 1] : 0.0) + x - loc;  // mass before this thread's values
    if (acc < goal && acc + loc >= goal) {
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        acc += v[k];
        if (acc >= goal) {
          atomicMin(&s_rank, tid * PER + k);
          break;
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    const int r = s_rank;
    const double q = (r + 1.0) / SAMPLE_N;
    const int delta = (int)(4.0 * sqrt(SAMPLE_N * q * (1.0 - q)) + 16.0) * 2;
    const int rh = r - delta, rl = r + delta;
    // inverted patterns: a smaller value is a larger probability
    ctl->win_hi = rh <= 0 ? 0x7ff0000000000000ull : ~(((uint64_t)a[rh] << 31) | (1ull << 63));
    ctl->win_lo = rl >= SAMPLE_N - 1 ? 0ull : ~((((uint64_t)a[rl] << 31) | (1ull << 63)) | 0x7fffffffull);
  }
}

constexpr int WP_BLOCK = 256, WP_ITEMS = 8;
static_assert(WP_BLOCK * WP_ITEMS == WINDOW_TILE, "window tiling");
constexpr int WP_TILE = WP_BLOCK * WP_ITEMS;

// One streaming pass over all terms (tile t = terms [t*WP_TILE, ...),
// static assignment): the exact fixed-point total mass, the count and mass
// above the window, the window's mass and its terms (probability, index)
// gathered into the window buffer, and per tile the number of terms above
// the window (they are kept whatever the exact cut is).
// Window terms are staged in shared memory and written out in batches, one
// atomic reservation per batch (a reservation per tile contended on a single
// counter); a tile with more window terms than the stage holds writes them
// directly.  The order of the window buffer is immaterial (the select works
// on values, the tile counts on indices).
constexpr int WP_STAGE = 1024;

struct WindowStage {
  uint64_t p[WP_STAGE];
  uint32_t i[WP_STAGE];
  uint32_t n;
  uint64_t base;
};

// With SUM the flushing threads also add the masses of the terms they copy
// (the window mass of the pass with a known total).
template <bool SUM>
__device__ __forceinline__ void window_flush(WindowStage& st, Ctl* ctl, uint64_t* __restrict__ wp,
                                             uint32_t* __restrict__ wi, uint64_t cap, u128& wsum) {
  // all threads call it; st.n is block-uniform
  const uint32_t cnt = st.n;
  if (cnt == 0) return;
  if (threadIdx.x == 0) st.base = atomicAdd((unsigned long long*)&ctl->win_n, (unsigned long long)cnt);
  __syncthreads();
  const uint64_t b = st.base;
  for (uint32_t j = threadIdx.x; j < cnt; j += WP_BLOCK) {
    const uint64_t o = b + j;
    if (SUM) wsum += fx_from_bits(st.p[j], &ctl->err);
    if (o < cap) {
      wp[o] = st.p[j];
      wi[o] = st.i[j];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) st.n = 0;
  __syncthreads();
}

// MODE (how the exact masses are summed):
//   WP_FULL  every term converted: the total, above-window and window masses;
//   WP_ABOVE a top-K cut with the total already known (summed by the gate):
//            only the masses above the window, from a per-warp queue of their
//            probabilities, so the 128-bit conversions run on full warps of
//            above-window terms only;
//   WP_BELOW a p-mass cut with the total known: the window and below-window
//            masses (the window terms converted while they are written out,
//            the others through the queue); the mass above the window is the
//            total minus those two, formed exactly by the decision kernel.
//            At p near 1 the window sits in the light tail, so few terms are
//            converted.
constexpr int WP_FULL = 0, WP_ABOVE = 1, WP_BELOW = 2;
template <int MODE>
__global__ void __launch_bounds__(WP_BLOCK, 4) k_window_pass(const uint64_t* __restrict__ probs,
                                                          uint64_t n, Ctl* ctl, uint64_t* __restrict__ wp,
                                                          uint32_t* __restrict__ wi,
                                                          uint64_t cap, uint32_t* __restrict__ tile_keep,
                                                          uint32_t* __restrict__ keep_bits) {
  pdl_prologue();
  typedef TileLayout<WP_BLOCK, WP_ITEMS> L;
  __shared__ uint32_t s_warp[WP_BLOCK / 32];
  __shared__ uint32_t s_above[WP_BLOCK / 32];
  __shared__ uint32_t s_acc;
  __shared__ uint64_t s_direct;
  __shared__ WindowStage st;
  constexpr bool QUEUE = MODE != WP_FULL;
  __shared__ uint64_t s_aq[QUEUE ? WP_BLOCK / 32 : 1][64];  // per-warp ring of probabilities to convert
  const uint64_t hi = ctl->win_hi, lo = ctl->win_lo;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  if (threadIdx.x == 0) st.n = 0;
  u128 tot = 0, above_m = 0, win_m = 0;  // WP_BELOW: above_m holds the mass below the window
  uint64_t above_c = 0, pmax = 0;
  uint32_t q_head = 0, q_n = 0;  // warp-uniform ring state
  const uint64_t tiles = (n + L::TILE - 1) / L::TILE;
  for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint64_t base = tile * L::TILE;
    // item j of this lane is term e0 + 32 j (TileLayout); rem: terms left from e0
    const uint64_t e0 = base + (uint64_t)warp * 32 * WP_ITEMS + lane;
    const int32_t rem = n > e0 ? (int32_t)min(n - e0, (uint64_t)(32 * WP_ITEMS)) : 0;
    uint64_t pbv[WP_ITEMS];
#pragma unroll
    for (int j = 0; j < WP_ITEMS; ++j) pbv[j] = 32 * j < rem ? probs[e0 + 32 * j] : 0ull;  // all loads first
    // the largest probability: with a top-K window (the cut inside it, so
    // the maximum is above it or in it) from the queued above-window terms
    // and the window terms only, else from every term (absent ones read 0)
    if (MODE != WP_ABOVE) {
#pragma unroll
      for (int j = 0; j < WP_ITEMS; ++j) pmax = pbv[j] > pmax ? pbv[j] : pmax;
    }
    uint32_t wmask = 0, run = 0, tile_above = 0;
    if (QUEUE) {
      // tile_above and run are warp-wide counts (the same in every lane);
      // lane j keeps item j's keep-flag word (one flag per term above the
      // window: kept whatever the exact cut; window terms kept by the cut are
      // added later), stored once per warp
      uint32_t kbits = 0;
#pragma unroll
      for (int j = 0; j < WP_ITEMS; ++j) {
        const uint64_t pb = pbv[j];
        const bool valid = 32 * j < rem;
        const bool above = valid && pb > hi;
        const bool inwin = valid && !above && pb >= lo;
        const bool queued = MODE == WP_ABOVE ? above : (valid && !above && !inwin);
        const uint32_t ab = __ballot_sync(0xffffffffu, above);
        const uint32_t qb = MODE == WP_ABOVE ? ab : __ballot_sync(0xffffffffu, queued);
        if (lane == j) kbits = ab;
        tile_above += (uint32_t)__popc(ab);
        if (queued) s_aq[warp][(q_head + q_n + __popc(qb & lt)) & 63u] = pb;
        q_n += __popc(qb);
        if (q_n >= 32) {  // a full warp of queued terms: one conversion each
          __syncwarp();
          const uint64_t qp = s_aq[warp][(q_head + lane) & 63u];
          above_m += fx_from_bits(qp, &ctl->err);
          if (MODE == WP_ABOVE) pmax = qp > pmax ? qp : pmax;
          __syncwarp();
          q_head = (q_head + 32) & 63u;
          q_n -= 32;
        }
        if (inwin) wmask |= 1u << j;
        run += __popc(__ballot_sync(0xffffffffu, inwin));
      }
      const uint64_t row0 = (base + (uint64_t)warp * 32 * WP_ITEMS) >> 5;
      if (lane < WP_ITEMS && ((row0 + lane) << 5) < n) keep_bits[row0 + lane] = kbits;
      if (lane == 0) above_c += tile_above;
    } else {
#pragma unroll
      for (int j = 0; j < WP_ITEMS; ++j) {
        const uint64_t pb = pbv[j];
        const bool valid = 32 * j < rem;
        const bool above = valid && pb > hi;
        const bool inwin = valid && !above && pb >= lo;
        const u128 f = fx_from_bits(pb, &ctl->err);
        tot += f;
        if (above) {
          ++tile_above;
          above_m += f;
        }
        if (inwin) {
          win_m += f;
          wmask |= 1u << j;
        }
        run += __popc(__ballot_sync(0xffffffffu, inwin));
        // terms above the window are kept whatever the exact cut: one flag
        // word per 32 consecutive terms (window terms kept by the cut are
        // added later)
        const uint32_t kb = __ballot_sync(0xffffffffu, above);
        if (lane == 0 && 32 * j < rem) keep_bits[(e0 >> 5) + j] = kb;  // lane 0: e0 starts a 32-term row
      }
      above_c += tile_above;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tile_above += __shfl_xor_sync(0xffffffffu, tile_above, o);
    }
    if (lane == 0) {
      s_warp[warp] = run;
      s_above[warp] = tile_above;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t acc = 0, ab = 0;
      for (int w = 0; w < WP_BLOCK / 32; ++w) {
        uint32_t c = s_warp[w];
        s_warp[w] = acc;
        acc += c;
        ab += s_above[w];
      }
      tile_keep[tile] = ab;
      s_acc = acc;
      s_direct = acc > WP_STAGE ? atomicAdd((unsigned long long*)&ctl->win_n, (unsigned long long)acc) : 0ull;
    }
    __syncthreads();
    const uint32_t acc = s_acc;
    if (acc == 0) continue;  // block-uniform
    const bool direct = acc > WP_STAGE;
    if (!direct && st.n + acc > WP_STAGE) window_flush<MODE == WP_BELOW>(st, ctl, wp, wi, cap, win_m);
    const uint32_t sbase = st.n;
    uint32_t wrun = 0;  // window positions: the same ballots again, in item order
#pragma unroll
    for (int j = 0; j < WP_ITEMS; ++j) {
      const bool inwin = (wmask >> j) & 1u;
      const uint32_t b = __ballot_sync(0xffffffffu, inwin);
      const uint32_t wpos = s_warp[warp] + wrun + __popc(b & lt);
      wrun += __popc(b);
      if (inwin) {
        const uint64_t i = e0 + 32 * j;
        if (MODE == WP_ABOVE) pmax = pbv[j] > pmax ? pbv[j] : pmax;
        if (direct) {
          if (MODE == WP_BELOW) win_m += fx_from_bits(pbv[j], &ctl->err);
          const uint64_t o = s_direct + wpos;
          if (o < cap) {
            wp[o] = pbv[j];
            wi[o] = (uint32_t)i;
          }
        } else {
          st.p[sbase + wpos] = pbv[j];
          st.i[sbase + wpos] = (uint32_t)i;
        }
      }
    }
    __syncthreads();
    if (!direct && threadIdx.x == 0) st.n = sbase + acc;
    __syncthreads();
  }
  window_flush<MODE == WP_BELOW>(st, ctl, wp, wi, cap, win_m);
  if (QUEUE) {  // the queue's rest
    __syncwarp();
    if ((uint32_t)lane < q_n) {
      const uint64_t qp = s_aq[warp][(q_head + lane) & 63u];
      above_m += fx_from_bits(qp, &ctl->err);
      if (MODE == WP_ABOVE) pmax = qp > pmax ? qp : pmax;
    }
  }
  tot = warp_sum_u128(tot);
  above_m = warp_sum_u128(above_m);
  win_m = warp_sum_u128(win_m);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    above_c += __shfl_xor_sync(0xffffffffu, (unsigned long long)above_c, o);
    const uint64_t x = __shfl_xor_sync(0xffffffffu, (unsigned long long)pmax, o);
    pmax = x > pmax ? x : pmax;
  }
  if (lane == 0) {
    if (pmax) atomicMax((unsigned long long*)&ctl->pmax_bits, (unsigned long long)pmax);
    if (MODE == WP_FULL) atomic_add_u128(&ctl->total_mass_hi, &ctl->total_mass_lo, tot);
    if (MODE == WP_BELOW)
      atomic_add_u128(&ctl->below_mass_hi, &ctl->below_mass_lo, above_m);
    else
      atomic_add_u128(&ctl->above_mass_hi, &ctl->above_mass_lo, above_m);
    atomic_add_u128(&ctl->win_mass_hi, &ctl->win_mass_lo, win_m);
    atomicAdd((unsigned long long*)&ctl->above_count, (unsigned long long)above_c);
  }
}

// One thread: choose between the window and the full list and set up the
// select state (target from the exact total mass).
__global__ void k_window_decide(Ctl* ctl, int mode, uint64_t count_target, double p, uint64_t cap, uint64_t n,
                                int pass_mode) {
  pdl_prologue();
  const u128 total = make_u128(ctl->total_mass_hi, ctl->total_mass_lo);
  if (pass_mode == WP_BELOW) {  // the mass above the window: the total less the window and below it
    const u128 am = total - make_u128(ctl->win_mass_hi, ctl->win_mass_lo) -
                    make_u128(ctl->below_mass_hi, ctl->below_mass_lo);
    ctl->above_mass_hi = (uint64_t)(am >> 64);
    ctl->above_mass_lo = (uint64_t)am;
  }
  u128 target;
  if (mode == 0) {
    double T = __dmul_rn(p, fx_to_double(total));
    target = fx_from_bits((uint64_t)__double_as_longlong(T), &ctl->err);
  } else {
    target = (u128)count_target;
  }
  const u128 am = make_u128(ctl->above_mass_hi, ctl->above_mass_lo);
  const u128 wm = make_u128(ctl->win_mass_hi, ctl->win_mass_lo);
  const uint64_t ac = ctl->above_count, wn = ctl->win_n;
  bool valid = wn <= cap && wn > 0;
  if (mode == 1) valid = valid && (u128)ac < target && target <= (u128)(ac + wn);
  else valid = valid && am < target && target <= am + wm;
  // Every window term has ~prob in [~hi, ~lo], so all share the common
  // leading bits of those two patterns: the select starts below them.
  uint64_t zh = ~ctl->win_hi, zl = ~ctl->win_lo;
  int common = valid ? __clzll((long long)(zh ^ zl)) : 1;
  if (common < 1) common = 1;
  if (common > 64) common = 64;
  ctl->sel_prefix_hi = common >= 64 ? zh : (zh & ~((~0ull) >> common));
  ctl->sel_prefix_lo = 0;
  ctl->sel_bits = (uint32_t)common;
  ctl->sel_mode = (uint32_t)mode;
  ctl->sel_done = 0;
  ctl->sel_target_hi = (uint64_t)(target >> 64);
  ctl->sel_target_lo = (uint64_t)target;
  ctl->compact_n = 0;
  ctl->sel_gated = 1;  // the levels enqueued behind the window test on the device whether to run
  ctl->use_window = valid ? 1u : 0u;
  ctl->sel_before_count = valid ? ac : 0;
  ctl->sel_before_mass_hi = valid ? ctl->above_mass_hi : 0;
  ctl->sel_before_mass_lo = valid ? ctl->above_mass_lo : 0;
  ctl->sel_bin_count = valid ? wn : n;
}

constexpr size_t SAMPLE_SMEM = 4 * (2 * SAMPLE_N + 32 * 256) + 8 * SAMPLE_THREADS;

static cudaError_t finish_attr();

cudaError_t select_prepare() {
  static DeviceOnce once;
  return once.run([] {
    cudaError_t e = cudaFuncSetAttribute(k_sample_window, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SAMPLE_SMEM);
    return e == cudaSuccess ? finish_attr() : e;
  });
}

void launch_select_window(const uint64_t* probs, const uint64_t* keys, uint64_t n, Ctl* ctl,
                          const SelectScratch& ss, int mode, uint64_t count_target, double p,
                          bool have_total, cudaStream_t st) {
  // with the total known (summed by the gate, or by the pass of an earlier
  // select on the same terms) the pass converts only the smaller side
  const int pmode = !have_total ? WP_FULL : (mode == 1 ? WP_ABOVE : WP_BELOW);
  const size_t smem = SAMPLE_SMEM;
  // the handle's creation checked the set-up on this device; without it the
  // launch fails and the next wait reports the launch error
  (void)select_prepare();
  launch_pdl(k_sample_window, 1, SAMPLE_THREADS, smem, st, probs, n, ctl, mode, count_target, p, have_total);
  uint64_t tiles = (n + WP_TILE - 1) / WP_TILE;
  uint64_t grid = tiles < 148 * 8 ? tiles : 148 * 8;
  if (grid == 0) grid = 1;
  if (pmode == WP_ABOVE)
    launch_pdl(k_window_pass<WP_ABOVE>, (unsigned)grid, WP_BLOCK, 0, st, probs, n, ctl, ss.win_p, ss.win_i,
               ss.win_cap, ss.tile_keep, ss.keep_bits);
  else if (pmode == WP_BELOW)
    launch_pdl(k_window_pass<WP_BELOW>, (unsigned)grid, WP_BLOCK, 0, st, probs, n, ctl, ss.win_p, ss.win_i,
               ss.win_cap, ss.tile_keep, ss.keep_bits);
  else
    launch_pdl(k_window_pass<WP_FULL>, (unsigned)grid, WP_BLOCK, 0, st, probs, n, ctl, ss.win_p, ss.win_i,
               ss.win_cap, ss.tile_keep, ss.keep_bits);
  launch_pdl(k_window_decide, 1, 1, 0, st, ctl, mode, count_target, p, ss.win_cap, n, pmode);
}

uint64_t window_tiles(uint64_t n) { return (n + WP_TILE - 1) / WP_TILE; }

// ---------------------------------------------------------------- windowed compaction
// After a select on the window: every tile's kept count is its count above
// the window plus its window terms not after the cut.
__global__ void k_window_tile_counts(const uint64_t* __restrict__ wp, const uint64_t* __restrict__ keys,
                                     const uint32_t* __restrict__ wi, Ctl* ctl,
                                     uint32_t* __restrict__ tile_keep, uint32_t* __restrict__ keep_bits) {
  pdl_prologue();
  const uint64_t wn = ctl->win_n;
  const uint64_t pc = ctl->cut_pbits, kc = ctl->cut_key;
  const int lane = threadIdx.x & 31;
  // warp-uniform loop: the window buffer is filled tile by tile per block,
  // so a warp's kept terms mostly share a tile: one count atomic per tile
  for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); b < wn;
       b += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j = b + lane;
    bool kept = false;
    uint32_t i = 0;
    if (j < wn) {
      const uint64_t pb = wp[j];
      i = wi[j];
      kept = pb > pc || (pb == pc && natural_key(ctl->nat, keys[i]) <= kc);
    }
    const uint32_t tile = kept ? i / WP_TILE : 0xffffffffu;
    const uint32_t peers = __match_any_sync(0xffffffffu, tile);
    if (kept) {
      if (lane == __ffs(peers) - 1) atomicAdd(&tile_keep[tile], (uint32_t)__popc(peers));
      atomicOr(&keep_bits[i >> 5], 1u << (i & 31));
    }
  }
}

// Exclusive scan of the per-tile kept counts by one block: each thread takes
// 8 consecutive tiles per round (loads first), one block scan per round.
// Thread 0 also sets the renormalisation scale 1/sqrt(S_c) of the cut.
constexpr int TS_ITEMS = 8;
__global__ void __launch_bounds__(1024) k_tile_scan(const uint32_t* __restrict__ tile_keep, uint64_t tiles,
                                                    uint64_t* __restrict__ tile_off, Ctl* ctl) {
  pdl_prologue();
  __shared__ uint64_t wsum[32];
  __shared__ uint64_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_carry = 0;
    const double sc = fx_to_double(make_u128(ctl->cut_mass_hi, ctl->cut_mass_lo));
    const double scale = __ddiv_rn(1.0, __dsqrt_rn(sc));
    ctl->scale = scale;
    // the largest probability is always kept; after the rescale it is about
    // pmax s^2, and a kept term whose larger |component| x' has
    // 2 x'^2 (1 + eps) below that cannot be the peak (eps covers the
    // roundings of both precisions' rescale and probability: 2^-20 for the
    // complex64 float rescale, far above them)
    const double pmax = __longlong_as_double((long long)ctl->pmax_bits);
    ctl->peak_thr = __dmul_rn(__dmul_rn(__dsqrt_rn(__dmul_rn(pmax, 0.5)), scale), 1.0 - 0x1p-20);
  }
  __syncthreads();
  for (uint64_t b0 = 0; b0 < tiles; b0 += 1024 * TS_ITEMS) {
    const uint64_t t0 = b0 + (uint64_t)threadIdx.x * TS_ITEMS;
    uint32_t v[TS_ITEMS];
#pragma unroll
    for (int j = 0; j < TS_ITEMS; ++j) v[j] = t0 + j < tiles ? tile_keep[t0 + j] : 0u;
    uint64_t sum = 0;
#pragma unroll
    for (int j = 0; j < TS_ITEMS; ++j) sum += v[j];
    uint64_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, (unsigned long long)x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint64_t y = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t z = __shfl_up_sync(0xffffffffu, (unsigned long long)y, o);
        if (lane >= o) y += z;
      }
      wsum[lane] = y;  // inclusive over the warps
    }
    __syncthreads();
    uint64_t o = s_carry + (warp > 0 ? wsum[warp - 1] : 0ull) + x - sum;
#pragma unroll
    for (int j = 0; j < TS_ITEMS; ++j) {
      if (t0 + j < tiles) tile_off[t0 + j] = o;
      o += v[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) s_carry += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) ctl->count[2] = s_carry;
}

// ---------------------------------------------------------------- pick
constexpr int PICK_THREADS = 1024;

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

__global__ void __launch_bounds__(PICK_THREADS) k_select_pick(Ctl* ctl, uint32_t* cnt, uint64_t* mass, double p) {
  pdl_prologue();
  if (ctl->sel_done) return;  // the level's histogram kernel added nothing either
  if (ctl->sel_gated && ctl->sel_bin_count <= (uint64_t)FINISH_CAP) return;
  block_pick(cnt, mass, ctl, p);  // ends with a block barrier
  for (int i = threadIdx.x; i < SEL_BINS; i += PICK_THREADS) {  // cleared for the next level
    cnt[i] = 0;
    mass[2 * i] = mass[2 * i + 1] = 0;
  }
}

void launch_select_pick(Ctl* ctl, const SelectScratch& ss, double p, cudaStream_t st) {
  launch_pdl(k_select_pick, 1, PICK_THREADS, 0, st, ctl, ss.hist_count, ss.hist_mass, p);
}

// ---------------------------------------------------------------- gather + finish
__global__ void __launch_bounds__(256) k_select_compact(const uint64_t* __restrict__ probs,
                                                        const uint64_t* __restrict__ keys, uint64_t n,
                                                        const uint64_t* __restrict__ wp,
                                                        const uint32_t* __restrict__ wi, Ctl* ctl,
                                                        uint64_t* __restrict__ buf) {
  pdl_prologue();
  if (ctl->sel_done) return;
  if (ctl->sel_gated && ctl->sel_bin_count > (uint64_t)FINISH_CAP) return;  // more levels first
  const bool win = ctl->use_window != 0;
  const uint64_t* P = win ? wp : probs;
  const uint64_t nn = win ? ctl->win_n : n;
  const int bits = (int)ctl->sel_bits;
  const uint64_t ph = ctl->sel_prefix_hi, pl = ctl->sel_prefix_lo;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nn;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t hi = ~P[i];
    if (bits <= 64 && ((hi ^ ph) >> (64 - bits)) != 0) continue;
    uint64_t lo = natural_key(ctl->nat, keys[win ? (uint64_t)wi[i] : i]);
    if (!z_matches(hi, lo, ph, pl, bits)) continue;
    uint64_t pos = atomicAdd((unsigned long long*)&ctl->compact_n, 1ull);
    if (pos < FINISH_CAP) {
      buf[2 * pos] = hi;
      buf[2 * pos + 1] = lo;
    }
  }
}

// ctl->compact_n arrives cleared (by the window's decision or the last finish).
void launch_select_compact(const uint64_t* probs, const uint64_t* keys, uint64_t n, Ctl* ctl,
                           const SelectScratch& ss, cudaStream_t st) {
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 4) blocks = 148 * 4;
  launch_pdl(k_select_compact, (unsigned)blocks, 256, 0, st, probs, keys, n, ss.win_p, ss.win_i, ctl, ss.buf);
}

// The chosen bin's terms (at most FINISH_CAP, gathered by k_select_compact)
// are sorted in shared memory by Z (a bitonic network over the next power of
// two, padded with the largest Z), their exact masses prefix-summed in that
// order, and the cut is the first of them where the running count or mass
// (after the terms before the bin) reaches the target -- the same term the
// radix levels would isolate, found without further levels (ties on the
// probability, common in states with equal-magnitude amplitudes, cost no
// extra passes).
constexpr size_t FINISH_SMEM = sizeof(uint64_t) * 2 * FINISH_CAP;

__global__ void __launch_bounds__(PICK_THREADS) k_select_finish(Ctl* ctl, const uint64_t* buf,
                                                                double p) {
  pdl_prologue();
  (void)p;
  extern __shared__ __align__(16) uint8_t s_dyn[];
  uint64_t* zh = reinterpret_cast<uint64_t*>(s_dyn);
  uint64_t* zl = zh + FINISH_CAP;
  __shared__ u128 w_m[PICK_THREADS / 32];
  __shared__ uint32_t s_first;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool gated = ctl->sel_gated != 0;
  const bool done = ctl->sel_done != 0;
  const uint64_t bin0 = ctl->sel_bin_count;
  uint64_t nb = ctl->compact_n;
  __syncthreads();
  if (tid == 0) {  // the gated run ends here; the next gather starts from an empty buffer
    ctl->sel_gated = 0;
    ctl->compact_n = 0;
  }
  if (done || (gated && bin0 > (uint64_t)FINISH_CAP)) return;
  if (nb > FINISH_CAP) nb = FINISH_CAP;
  uint32_t n2 = 1;
  while (n2 < nb) n2 <<= 1;
  for (uint32_t i = tid; i < n2; i += PICK_THREADS) {
    const bool real = i < nb;
    zh[i] = real ? buf[2 * i] : ~0ull;
    zl[i] = real ? buf[2 * i + 1] : ~0ull;
  }
  __syncthreads();
  for (uint32_t k = 2; k <= n2; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t t = tid; t < n2 / 2; t += PICK_THREADS) {
        const uint32_t i = 2 * t - (t & (j - 1));  // bit j of i clear; its partner is i + j
        const uint32_t l = i + j;
        const uint64_t ah = zh[i], al = zl[i], bh = zh[l], bl = zl[l];
        const bool gt = ah > bh || (ah == bh && al > bl);
        if (gt == ((i & k) == 0)) {  // ascending where bit k of i is clear
          zh[i] = bh;
          zl[i] = bl;
          zh[l] = ah;
          zl[l] = al;
        }
      }
      __syncthreads();
    }
  }
  // each thread a contiguous run of the sorted terms: exact masses scanned
  const uint32_t per = (n2 + PICK_THREADS - 1) / PICK_THREADS;
  const uint32_t b0 = (uint32_t)tid * per;
  u128 my = 0;
  for (uint32_t i = b0; i < b0 + per && i < nb; ++i) my += fx_from_bits(~zh[i], &ctl->err);
  u128 x = my;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u128 y = shfl_up_u128(x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) w_m[warp] = x;
  if (tid == 0) s_first = 0xffffffffu;
  __syncthreads();
  u128 base = 0;
  for (int w = 0; w < warp; ++w) base += w_m[w];
  const uint32_t mode = ctl->sel_mode;
  const u128 target = make_u128(ctl->sel_target_hi, ctl->sel_target_lo);
  const uint64_t before_c = ctl->sel_before_count;
  const u128 before_m = make_u128(ctl->sel_before_mass_hi, ctl->sel_before_mass_lo) + base + x - my;
  {
    u128 cm = before_m;
    for (uint32_t i = b0; i < b0 + per && i < nb; ++i) {
      cm += fx_from_bits(~zh[i], &ctl->err);
      if (mode == 1 ? (u128)(before_c + i + 1) >= target : cm >= target) {
        atomicMin(&s_first, i);
        break;
      }
    }
  }
  __syncthreads();
  const uint32_t first = s_first;
  if (first == 0xffffffffu) {
    if (tid == 0) ctl->sel_done = 2;  // the target is never reached: no cut
    return;
  }
  if (first >= b0 && first < b0 + per) {
    u128 sc = before_m;
    for (uint32_t i = b0; i <= first; ++i) sc += fx_from_bits(~zh[i], &ctl->err);
    ctl->cut_pbits = ~zh[first];
    ctl->cut_key = zl[first];
    ctl->cut_count = before_c + first + 1;
    ctl->cut_mass_hi = (uint64_t)(sc >> 64);
    ctl->cut_mass_lo = (uint64_t)sc;
    ctl->sel_done = 1;
  }
}

static cudaError_t finish_attr() {
  return cudaFuncSetAttribute(k_select_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FINISH_SMEM);
}

void launch_select_finish(Ctl* ctl, const SelectScratch& ss, double p, cudaStream_t st) {
  (void)select_prepare();  // checked at the handle's creation
  launch_pdl(k_select_finish, 1, PICK_THREADS, FINISH_SMEM, st, ctl, ss.buf, p);
}

// ---------------------------------------------------------------- peak partials
// The compactions keep each block's canonical best kept term (probability
// bits larger, then key smaller), so the peak readout after a truncation
// reduces these partials instead of reading the state again.
__device__ __forceinline__ void peak_take(uint64_t& bp, uint64_t& bk, uint64_t p, uint64_t k) {
  if (p > bp || (p == bp && k < bk)) {
    bp = p;
    bk = k;
  }
}

// A thread's best kept term while it writes stored keys: the stored key of
// the best is kept and made natural once at the end; only exact probability
// ties compare natural keys on the way.
struct PeakRun {
  uint64_t p = 0, k = 0;
  bool any = false;
  __device__ __forceinline__ void take(uint64_t pb, uint64_t key, const uint64_t* nat) {
    if (!any || pb > p) {
      p = pb;
      k = key;
      any = true;
    } else if (pb == p && natural_key(nat, key) < natural_key(nat, k)) {
      k = key;
    }
  }
  __device__ __forceinline__ uint64_t natural(const uint64_t* nat) const { return any ? natural_key(nat, k) : ~0ull; }
};

// The windowed compaction rescales every kept term but needs the new
// probability only of terms that can be the peak: with the largest
// probability pmax (always kept) taken by the window pass, a term whose
// larger |component| after the rescale lies below peak_thr (about
// sqrt(pmax / 2) s, see k_tile_scan) is less probable than that term.  The
// test is one integer compare on the component bits, so whole warps skip
// the FP64 work together (the threshold is the same in every lane).
__device__ __forceinline__ uint64_t peak_abs_bits(double2 a) {
  const uint64_t x = (uint64_t)__double_as_longlong(a.x) & 0x7fffffffffffffffull;
  const uint64_t y = (uint64_t)__double_as_longlong(a.y) & 0x7fffffffffffffffull;
  return x > y ? x : y;
}
__device__ __forceinline__ uint64_t peak_abs_bits(float2 a) {
  const uint32_t x = __float_as_uint(a.x) & 0x7fffffffu, y = __float_as_uint(a.y) & 0x7fffffffu;
  return x > y ? x : y;
}
// peak_thr as bits of the amplitude's precision (rounded down for float).
template <typename C2>
__device__ __forceinline__ uint64_t peak_thr_bits(double t) {
  if (sizeof(C2) == sizeof(double2)) return (uint64_t)__double_as_longlong(t);
  return (uint64_t)__float_as_uint(__double2float_rd(t));
}

// Block-wide best of (bp, bk) into out[0] (probability bits), out[1] (key);
// all threads must call it.
__device__ void block_peak_write(uint64_t bp, uint64_t bk, uint64_t* out) {
  __shared__ uint64_t s_p[32], s_k[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t p2 = __shfl_down_sync(0xffffffffu, (unsigned long long)bp, o);
    const uint64_t k2 = __shfl_down_sync(0xffffffffu, (unsigned long long)bk, o);
    peak_take(bp, bk, p2, k2);
  }
  if (lane == 0) {
    s_p[warp] = bp;
    s_k[warp] = bk;
  }
  __syncthreads();
  if (warp == 0) {
    bp = lane < warps ? s_p[lane] : 0ull;
    bk = lane < warps ? s_k[lane] : ~0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t p2 = __shfl_down_sync(0xffffffffu, (unsigned long long)bp, o);
      const uint64_t k2 = __shfl_down_sync(0xffffffffu, (unsigned long long)bk, o);
      peak_take(bp, bk, p2, k2);
    }
    if (lane == 0) {
      out[0] = bp;
      out[1] = bk;
    }
  }
}

// Reduce the partials of the last compaction (n blocks) into ctl->peak_z_*.
__global__ void __launch_bounds__(256) k_peak_partials(const uint64_t* __restrict__ part, uint32_t n, Ctl* ctl) {
  pdl_prologue();
  uint64_t bp = 0, bk = ~0ull;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) peak_take(bp, bk, part[2 * i], part[2 * i + 1]);
  __shared__ uint64_t out[2];
  block_peak_write(bp, bk, out);
  if (threadIdx.x == 0) {
    ctl->peak_z_hi = out[0];
    ctl->peak_z_lo = out[1];
  }
}

void launch_peak_partials(const uint64_t* part, uint32_t n, Ctl* ctl, cudaStream_t st) {
  launch_pdl(k_peak_partials, 1, 256, 0, st, part, n, ctl);
}

// ---------------------------------------------------------------- compaction
__global__ void k_set_scale(Ctl* ctl) {
  pdl_prologue();
  double sc = fx_to_double(make_u128(ctl->cut_mass_hi, ctl->cut_mass_lo));
  ctl->scale = __ddiv_rn(1.0, __dsqrt_rn(sc));
}

void launch_set_scale(Ctl* ctl, cudaStream_t st) { launch_pdl(k_set_scale, 1, 1, 0, st, ctl); }

// Select state for one histogram level over all terms (no window, not gated).
__global__ void k_set_select(Ctl* ctl, uint64_t ph, uint64_t pl, uint32_t bits) {
  pdl_prologue();
  ctl->sel_prefix_hi = ph;
  ctl->sel_prefix_lo = pl;
  ctl->sel_bits = bits;
  ctl->sel_done = 0;
  ctl->sel_gated = 0;
  ctl->use_window = 0;
}

void launch_set_select(Ctl* ctl, uint64_t ph, uint64_t pl, uint32_t bits, cudaStream_t st) {
  launch_pdl(k_set_select, 1, 1, 0, st, ctl, ph, pl, bits);
}

// A cut given from outside: keep the terms not after the composite
// (~pc, kc) in canonical order; S_c = (sc_hi, sc_lo).
__global__ void k_set_cut(Ctl* ctl, uint64_t pc, uint64_t kc, uint64_t sc_hi, uint64_t sc_lo) {
  pdl_prologue();
  ctl->cut_pbits = pc;
  ctl->cut_key = kc;
  ctl->cut_mass_hi = sc_hi;
  ctl->cut_mass_lo = sc_lo;
}

void launch_set_cut(Ctl* ctl, uint64_t pc, uint64_t kc, uint64_t sc_hi, uint64_t sc_lo, cudaStream_t st) {
  launch_pdl(k_set_cut, 1, 1, 0, st, ctl, pc, kc, sc_hi, sc_lo);
}

constexpr int TC_BLOCK = 256, TC_ITEMS = 8;

// Keep the terms not after the cut (probability above the cut's, or equal
// with key not above it), in input order, scaled by ctl->scale.  Only the
// probability is read for every term; keys (for ties at the cut) and
// amplitudes are read for the kept terms.
template <typename C2>
__global__ void __launch_bounds__(TC_BLOCK) k_truncate_compact(
    const uint64_t* __restrict__ keys, const C2* __restrict__ amps, const uint64_t* __restrict__ probs,
    uint64_t n, uint64_t* __restrict__ keys_out, C2* __restrict__ amps_out, uint64_t* lookback, Ctl* ctl,
    uint64_t* __restrict__ peak_part) {
  typedef TileLayout<TC_BLOCK, TC_ITEMS> L;
  PeakRun best;
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
#pragma unroll
    for (int j = 0; j < TC_ITEMS; ++j) {
      const uint64_t i = L::index(base, j);
      bool f = false;
      if (i < n) {
        const uint64_t pb = probs[i];
        f = pb > pc || (pb == pc && natural_key(ctl->nat, keys[i]) <= kc);
      }
      flag[j] = f;
    }
    tile_compact<TC_BLOCK, TC_ITEMS>(flag, pos, cs, lookback, tile, &ctl->err);
#pragma unroll
    for (int j = 0; j < TC_ITEMS; ++j) {
      if (flag[j]) {
        const uint64_t i = L::index(base, j);
        const uint64_t o = cs.tile_base_out + pos[j];
        const C2 a = amp_scaled(amps[i], s);
        const uint64_t k = keys[i];
        keys_out[o] = k;
        amps_out[o] = a;
        best.take(amp_prob_bits(a), k, ctl->nat);
      }
    }
    if (tile == tiles - 1 && threadIdx.x == 0) ctl->count[2] = cs.tile_base_out + cs.tile_total;
    __syncthreads();
  }
  block_peak_write(best.p, best.natural(ctl->nat), peak_part + 2 * blockIdx.x);
}

// Windowed compaction: tile t (same tiling as the window pass) writes its
// kept terms from tile_off[t] on, in input order; no cross-tile waiting.
// The keep flags come from the window pass (terms above the window) and the
// window's own cut decisions, one bit per term, so only the kept terms' keys
// and amplitudes are read.
template <typename C2>
__global__ void __launch_bounds__(WP_BLOCK) k_truncate_write(
    const uint64_t* __restrict__ keys, const C2* __restrict__ amps, const uint32_t* __restrict__ keep_bits,
    uint64_t n, const uint64_t* __restrict__ tile_off, uint64_t* __restrict__ keys_out,
    C2* __restrict__ amps_out, const Ctl* ctl, uint64_t* __restrict__ peak_part) {
  pdl_prologue();
  typedef TileLayout<WP_BLOCK, WP_ITEMS> L;
  __shared__ CompactShared<WP_BLOCK> cs;
  __shared__ uint16_t s_list[WP_TILE];
  PeakRun best;
  const double s = ctl->scale;
  const uint64_t thr = peak_thr_bits<C2>(ctl->peak_thr);
  const uint64_t* nat = ctl->nat;
  const int lane = threadIdx.x & 31;
  const uint64_t tiles = (n + L::TILE - 1) / L::TILE;
  for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint64_t base = tile * L::TILE;
    uint32_t words[WP_ITEMS];
#pragma unroll
    for (int j = 0; j < WP_ITEMS; ++j) {
      const uint64_t row = L::index(base, j) - lane;
      words[j] = row < n ? keep_bits[row >> 5] : 0u;
    }
    bool flag[WP_ITEMS];
    uint32_t pos[WP_ITEMS];
#pragma unroll
    for (int j = 0; j < WP_ITEMS; ++j) flag[j] = L::index(base, j) < n && ((words[j] >> lane) & 1u);
    tile_local_positions<WP_BLOCK, WP_ITEMS>(flag, pos, cs);
    // list the kept terms (tile-local index, in input order), then process
    // the list densely: every lane does useful rescaling work and the
    // outputs are written contiguously
#pragma unroll
    for (int j = 0; j < WP_ITEMS; ++j)
      if (flag[j]) s_list[pos[j]] = (uint16_t)(L::index(base, j) - base);
    __syncthreads();
    const uint64_t ob = tile_off[tile];
    const uint32_t kept = cs.tile_total;
    constexpr int U = 4;  // kept terms per thread whose loads are issued together
    for (uint32_t t0 = threadIdx.x; t0 < kept; t0 += U * WP_BLOCK) {
      C2 a[U];
      uint64_t k[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t t = t0 + u * WP_BLOCK;
        if (t < kept) {
          const uint64_t i = base + s_list[t];
          a[u] = amps[i];
          k[u] = keys[i];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t t = t0 + u * WP_BLOCK;
        if (t < kept) {
          const C2 y = amp_scaled(a[u], s);
          keys_out[ob + t] = k[u];
          amps_out[ob + t] = y;
          if (peak_abs_bits(y) >= thr) best.take(amp_prob_bits(y), k[u], nat);
        }
      }
    }
    __syncthreads();
  }
  block_peak_write(best.p, best.natural(nat), peak_part + 2 * blockIdx.x);
}

void launch_truncate_windowed(int prec, const uint64_t* keys, const void* amps, const uint64_t* probs,
                              uint64_t n, uint64_t* keys_out, void* amps_out, const SelectScratch& ss, Ctl* ctl, cudaStream_t st, uint64_t* peak_part,
                              uint32_t* peak_blocks) {
  (void)probs;  // the keep flags replace the probabilities here
  const uint64_t tiles = window_tiles(n);
  launch_pdl(k_window_tile_counts, 148 * 4, 256, 0, st, ss.win_p, keys, ss.win_i, ctl, ss.tile_keep, ss.keep_bits);
  launch_pdl(k_tile_scan, 1, 1024, 0, st, ss.tile_keep, tiles, ss.tile_off, ctl);
  uint64_t grid = tiles < PEAK_PARTS ? tiles : PEAK_PARTS;
  if (grid == 0) grid = 1;
  *peak_blocks = (uint32_t)grid;
  if (prec == 0)
    launch_pdl(k_truncate_write<double2>, (unsigned)grid, WP_BLOCK, 0, st, keys, (const double2*)amps, ss.keep_bits,
               n, ss.tile_off, keys_out, (double2*)amps_out, ctl, peak_part);
  else
    launch_pdl(k_truncate_write<float2>, (unsigned)grid, WP_BLOCK, 0, st, keys, (const float2*)amps, ss.keep_bits,
               n, ss.tile_off, keys_out, (float2*)amps_out, ctl, peak_part);
}

void launch_truncate_compact(int prec, const uint64_t* keys, const void* amps, const uint64_t* probs,
                             uint64_t n, uint64_t* keys_out, void* amps_out, uint64_t* lookback, Ctl* ctl, cudaStream_t st, uint64_t* peak_part,
                             uint32_t* peak_blocks) {
  uint64_t tiles = (n + TC_BLOCK * TC_ITEMS - 1) / (TC_BLOCK * TC_ITEMS);
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * (tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[2], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[2], 0, sizeof(uint64_t), st);
  *peak_blocks = 0;
  if (n == 0) return;
  uint64_t grid = tiles < PEAK_PARTS ? tiles : PEAK_PARTS;
  *peak_blocks = (uint32_t)grid;
  if (prec == 0)
    k_truncate_compact<double2><<<(unsigned)grid, TC_BLOCK, 0, st>>>(
        keys, (const double2*)amps, probs, n, keys_out, (double2*)amps_out, lookback, ctl, peak_part);
  else
    k_truncate_compact<float2><<<(unsigned)grid, TC_BLOCK, 0, st>>>(
        keys, (const float2*)amps, probs, n, keys_out, (float2*)amps_out, lookback, ctl, peak_part);
}

// ---------------------------------------------------------------- probabilities
template <typename C2>
__global__ void k_amp_probs(const C2* __restrict__ amps, uint64_t n, uint64_t* __restrict__ probs) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    probs[i] = amp_prob_bits(amps[i]);
}

void launch_amp_probs(int prec, const void* amps, uint64_t n, uint64_t* probs, cudaStream_t st) {
  if (n == 0) return;
  const uint64_t blocks = (n + 255) / 256;
  const unsigned grid = (unsigned)(blocks < 148 * 8 ? blocks : 148 * 8);
  if (prec == 0) k_amp_probs<double2><<<grid, 256, 0, st>>>((const double2*)amps, n, probs);
  else k_amp_probs<float2><<<grid, 256, 0, st>>>((const float2*)amps, n, probs);
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
      const uint64_t k = natural_key(ctl->nat, keys[i]);
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
                               double2* __restrict__ amps_out, uint64_t* __restrict__ probs_out,
                               const Ctl* ctl) {
  const uint64_t* nat = ctl ? ctl->nat : nullptr;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t j = idx[i];
    if (keys_out) keys_out[i] = natural_key(nat, keys[j]);
    if (amps_out) {
      C2 a = amps[j];
      amps_out[i] = make_double2((double)a.x, (double)a.y);
    }
    if (probs_out) probs_out[i] = probs[j];
  }
}

void launch_gather_terms(int prec, const uint32_t* idx, uint64_t n, const uint64_t* keys,
                         const void* amps, const uint64_t* probs, uint64_t* keys_out,
                         double* amps_out, uint64_t* probs_out, const Ctl* ctl, cudaStream_t st) {
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  if (prec == 0)
    k_gather_terms<double2><<<(unsigned)blocks, 256, 0, st>>>(
        idx, n, keys, (const double2*)amps, probs, keys_out, (double2*)amps_out, probs_out, ctl);
  else
    k_gather_terms<float2><<<(unsigned)blocks, 256, 0, st>>>(
        idx, n, keys, (const float2*)amps, probs, keys_out, (double2*)amps_out, probs_out, ctl);
}

__global__ void k_keys_natural(const uint64_t* __restrict__ keys, uint64_t n, const Ctl* ctl,
                               uint64_t* __restrict__ out) {
  const uint64_t* nat = ctl->nat;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = natural_key(nat, keys[i]);
}

void launch_keys_natural(const uint64_t* keys, uint64_t n, const Ctl* ctl, uint64_t* out, cudaStream_t st) {
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_keys_natural<<<(unsigned)blocks, 256, 0, st>>>(keys, n, ctl, out);
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
        probs_out[o] = amp_prob_bits(av[j]);
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
