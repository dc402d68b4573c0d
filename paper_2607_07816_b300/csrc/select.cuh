// Radix-select helpers shared by the single-state and batched selects: the
// select key z = (~prob_bits, key) as 128 bits, digit positions, prefix
// tests and the warp-aggregated (count, fixed-point mass) histogram add.
#pragma once
#include "common.cuh"
#include "internal.h"

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

// Adds one element per lane to the shared histograms.  Lanes with the same
// digit are merged first (__match_any_sync): the lowest lane of each group
// adds the group's count and mass, so a hot bin takes one atomic per warp
// instead of one per element.  All lanes of a bin share the probability's
// exponent (the exponent is fixed before any other bits), so the group mass
// is the exact sum of the mantissas times a common power of two; the
// mantissa sum is formed by three 18-bit chunked warp reductions (no chunk
// sum can exceed 32 bits).  Probabilities below 2^-68, whose fixed-point
// value is a truncated shift, and those of 2 or more (whose group sum could
// exceed 128 bits) are added one by one.
__device__ __forceinline__ void warp_hist_add(bool active, uint32_t dg, uint64_t pb, uint32_t* cnt,
                                              uint64_t* mass, uint32_t* err) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t key = active ? dg : 0xffffffffu;
  const uint32_t peers = __match_any_sync(0xffffffffu, key);
  const uint32_t e = (uint32_t)(pb >> 52) & 0x7ffu;
  const int sh = (int)e - 955;
  const bool exact_shift = active && e != 0 && sh >= 0 && sh <= 68;
  uint64_t mant = exact_shift ? ((pb & ((1ull << 52) - 1)) | (1ull << 52)) : 0ull;
  const uint32_t s0 = __reduce_add_sync(peers, (uint32_t)(mant & 0x3ffffull));
  const uint32_t s1 = __reduce_add_sync(peers, (uint32_t)((mant >> 18) & 0x3ffffull));
  const uint32_t s2 = __reduce_add_sync(peers, (uint32_t)(mant >> 36));
  if (!active) return;
  if (lane == (uint32_t)(__ffs(peers) - 1)) {
    atomicAdd(&cnt[dg], (uint32_t)__popc(peers));
    const uint64_t msum = (uint64_t)s0 + ((uint64_t)s1 << 18) + ((uint64_t)s2 << 36);
    if (msum) atomic_add_u128(&mass[2 * dg], &mass[2 * dg + 1], ((u128)msum) << sh);
  }
  if (active && !exact_shift && e != 0) {  // tiny (or above 2) probability: added alone
    u128 v = fx_from_bits(pb, err);
    if (v) atomic_add_u128(&mass[2 * dg], &mass[2 * dg + 1], v);
  }
}

}  // namespace sv
