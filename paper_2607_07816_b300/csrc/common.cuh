// Device helpers shared by the kernels of libsv.so.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sv {

typedef unsigned __int128 u128;

// error bits recorded in the device control block
constexpr uint32_t ERR_TIMEOUT = 1u;   // a bounded spin-wait gave up
constexpr uint32_t ERR_MASS = 2u;      // a probability too large for the fixed-point mass
constexpr uint32_t ERR_INVARIANT = 4u; // duplicate keys reached a gate (groups larger than 2^m)
constexpr uint32_t ERR_BUCKET = 8u;    // a bucket exceeded the local-gate batch limit (recoverable)

// Bounded waits: a decoupled look-back poll gives up after this many polls
// (with exponential __nanosleep back-off capped at 256 ns: about a second).
constexpr uint32_t SPIN_LIMIT = 1u << 22;

// Look-back descriptor word: status in the top two bits, value below.
constexpr uint64_t LB_AGG = 1ull << 62;
constexpr uint64_t LB_INC = 2ull << 62;
constexpr uint64_t LB_VAL = (1ull << 62) - 1;

// Per-handle device control block.
struct Ctl {
  uint32_t err;
  uint32_t pad0;
  uint64_t tile_counter[4];   // dynamic tile ids for persistent kernels
  uint64_t count[4];          // produced counts (groups, candidates, kept, ...)
  // radix-select state (truncation)
  uint64_t sel_prefix_hi, sel_prefix_lo;   // composite bits fixed so far
  uint32_t sel_bits;                       // how many top bits are fixed
  uint32_t sel_mode;                       // 0 = by mass, 1 = by count
  uint32_t sel_done;
  uint32_t sel_compact;                    // next level also compacts matches
  uint64_t sel_target_hi, sel_target_lo;   // remaining mass / count target
  uint64_t sel_before_count;
  uint64_t sel_before_mass_hi, sel_before_mass_lo;
  uint64_t sel_bin_count;                  // count in the chosen bin
  uint64_t total_mass_hi, total_mass_lo;   // S_N
  uint64_t cut_count;                      // c (terms kept)
  uint64_t cut_mass_hi, cut_mass_lo;       // S_c
  uint64_t cut_pbits, cut_key;             // the c-th term in canonical order
  double scale;                            // 1/sqrt(double(S_c))
  uint64_t peak_z_hi, peak_z_lo;           // canonical composite of the peak
  uint64_t compact_n;                      // entries in the select buffer
  // sample-estimated window of the cut (truncation)
  uint64_t win_hi, win_lo;                 // window = probabilities in [lo, hi] (bit patterns)
  uint64_t win_n;                          // terms gathered into the window buffer
  uint64_t above_count;                    // terms with probability > hi
  uint64_t above_mass_hi, above_mass_lo;
  uint64_t win_mass_hi, win_mass_lo;
  uint64_t below_mass_hi, below_mass_lo;   // terms below the window (pass with a known total, by mass)
  uint32_t use_window;                     // 1: select over the window, 0: over all terms
  uint32_t sel_gated;                      // 1: select kernels decide on the device which of them run
  uint64_t kept_check;                     // terms the last truncation wrote (checked at the next wait)
  const uint64_t* nat;                     // natural-key table of the stored keys (null: keys are natural)
  uint64_t pmax_bits;                      // largest probability (bits) the window pass saw
  double peak_thr;                         // |component| below which a rescaled kept term cannot be the peak
};

__device__ __forceinline__ uint64_t ld_acquire(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Decoupled look-back (single-pass prefix scan, Merrill & Garland) over one
// chain, warp-cooperative: all 32 lanes of one warp call it.  The tile
// publishes its aggregate, then the warp polls a window of 32 predecessor
// descriptors at once, waits until every descriptor from the nearest
// inclusive prefix up to the tile is published, sums them with a warp
// reduction and moves the window back when it holds no inclusive prefix;
// finally the tile publishes its inclusive prefix.  Every lane returns the
// exclusive prefix.  Tiles obtain their ids in launch order from an atomic
// counter, so every tile waited on has already started; the wait is still
// bounded (spin_limit polls) and sets ERR_TIMEOUT instead of hanging.
__device__ __forceinline__ uint64_t lookback_exclusive_warp(uint64_t* lb, uint64_t tile, uint64_t agg,
                                                            uint32_t* err, uint32_t spin_limit = SPIN_LIMIT) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0) st_release(lb, LB_INC | agg);
    return 0;
  }
  if (lane == 0) st_release(lb + tile, LB_AGG | agg);
  uint64_t excl = 0;
  int64_t end = (int64_t)tile;  // window covers [end - 32, end)
  uint32_t spins = 0, ns = 8;
  while (true) {
    const int64_t t = end - 32 + lane;
    const uint64_t v = t >= 0 ? ld_acquire(lb + t) : LB_INC;  // before tile 0: an inclusive zero
    const uint32_t st = (uint32_t)(v >> 62);
    const uint32_t inc = __ballot_sync(0xffffffffu, st == 2u);
    const uint32_t notready = __ballot_sync(0xffffffffu, st == 0u);
    const int hi = inc ? 31 - __clz((int)inc) : 0;  // nearest inclusive prefix in the window
    const uint32_t need = inc ? (0xffffffffu << hi) : 0xffffffffu;
    if (notready & need) {
      if (++spins > spin_limit) {
        if (lane == 0) atomicOr(err, ERR_TIMEOUT);
        break;
      }
      __nanosleep(ns);
      if (ns < 256) ns <<= 1;
      continue;
    }
    uint64_t x = (lane >= hi) ? (v & LB_VAL) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, (unsigned long long)x, o);
    excl += x;
    if (inc) break;
    end -= 32;
  }
  if (lane == 0) st_release(lb + tile, LB_INC | (excl + agg));
  return excl;
}

__device__ __forceinline__ uint64_t shl64(uint64_t x, int s) { return s >= 64 ? 0ull : x << s; }
__device__ __forceinline__ uint64_t shr64(uint64_t x, int s) { return s >= 64 ? 0ull : x >> s; }
__device__ __forceinline__ uint64_t low_mask(int s) { return s >= 64 ? ~0ull : ((1ull << s) - 1); }

// Remove the bits at the ascending positions qs[0..m-1] from x (software
// bit-extract over the complement of the gate mask).
__device__ __forceinline__ uint64_t squeeze_out(uint64_t x, const int* qs, int m) {
#pragma unroll
  for (int t = 3; t >= 0; --t) {
    if (t < m) {
      int q = qs[t];
      x = (x & low_mask(q)) | shl64(shr64(x, q + 1), q);
    }
  }
  return x;
}

// Insert zero bits at the ascending positions qs[0..m-1] (inverse of
// squeeze_out on keys whose gate bits are zero).
__device__ __forceinline__ uint64_t spread_in(uint64_t x, const int* qs, int m) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (t < m) {
      int q = qs[t];
      x = (x & low_mask(q)) | shl64(shr64(x, q), q + 1);
    }
  }
  return x;
}

// A bit permutation of 64-bit keys as 16 nibble tables: the image of x is
// the OR of t[k][nibble k of x].
__device__ __forceinline__ uint64_t permute_bits(const uint64_t (*t)[16], uint64_t x) {
  uint64_t y = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) y |= t[k][(x >> (4 * k)) & 15u];
  return y;
}

// floor(p * 2^120) for the bit pattern b of a non-negative double p < 2^7.
// Larger values set ERR_MASS (the fixed-point sums would overflow).
__device__ __forceinline__ u128 fx_from_bits(uint64_t b, uint32_t* err) {
  uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
  if (e == 0) return 0;  // zero or subnormal: below 2^-1022, floors to 0
  uint64_t mant = (b & ((1ull << 52) - 1)) | (1ull << 52);
  int sh = (int)e - 955;  // p * 2^120 = mant * 2^(e - 1075 + 120)
  if (sh >= 0) {
    if (sh > 74) {
      atomicOr(err, ERR_MASS);
      return 0;
    }
    return ((u128)mant) << sh;
  }
  if (sh <= -64) return 0;
  return (u128)(mant >> (-sh));
}

// Nearest double (ties to even) to s * 2^-120.
__device__ __forceinline__ double fx_to_double(u128 s) {
  if (s == 0) return 0.0;
  uint64_t hi = (uint64_t)(s >> 64), lo = (uint64_t)s;
  int top = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
  int shift = top - 52;
  uint64_t m;
  if (shift <= 0) {
    m = lo;  // fewer than 54 significant bits: exact
    shift = 0;
  } else {
    u128 q = s >> shift;
    u128 rem = s - (q << shift);
    u128 half = ((u128)1) << (shift - 1);
    m = (uint64_t)q;
    if (rem > half || (rem == half && (m & 1ull))) ++m;  // may become 2^53: still exact
  }
  int k = shift - 120;  // value = m * 2^k, k in [-120, 8]
  double scale = __longlong_as_double((long long)((uint64_t)(1023 + k) << 52));
  return __ull2double_rn(m) * scale;
}

__device__ __forceinline__ u128 make_u128(uint64_t hi, uint64_t lo) { return ((u128)hi << 64) | lo; }

// prob = fma(re, re, im*im) in double (complex64 components are widened
// before the call, which makes both products exact).
__device__ __forceinline__ double prob_of(double re, double im) {
  return __fma_rn(re, re, __dmul_rn(im, im));
}

}  // namespace sv
