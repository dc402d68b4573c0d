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

__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(v >> 64), o);
    uint64_t lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)(uint64_t)v, o);
    v += make_u128(hi, lo);
  }
  return v;
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

// Digit of the first level (one bit fixed: the top bit of ~prob_bits, set
// for every non-negative probability) from a probability's bits.
__device__ __forceinline__ uint32_t sel_first_digit(uint64_t prob_bits) {
  return (uint32_t)(~prob_bits >> (63 - SEL_BITS)) & (SEL_BINS - 1u);
}

// Histogram adds with one bin's pending (count, exact fixed-point mass)
// held in each thread's registers: a thread touches the shared histogram only
// when its element falls into another bin than its last one.  A level whose
// elements fall into a few bins -- the first levels over a narrow window --
// then costs one shared atomic per thread and bin change instead of one per
// element on a few hot addresses (64-bit shared atomics on a hot address
// serialise).  Each thread flushes its cache before the block reads the
// histogram.
struct BinCache {
  uint32_t bin = 0xffffffffu;
  uint32_t cnt = 0;
  u128 mass = 0;
};

__device__ __forceinline__ void bin_cache_flush(BinCache& c, uint32_t* cnt, uint64_t* mass) {
  if (c.cnt) {
    atomicAdd(&cnt[c.bin], c.cnt);
    if (c.mass) atomic_add_u128(&mass[2 * c.bin], &mass[2 * c.bin + 1], c.mass);
  }
  c.cnt = 0;
  c.mass = 0;
}

__device__ __forceinline__ void hist_add(uint32_t dg, uint64_t pb, uint32_t* cnt, uint64_t* mass, uint32_t* err,
                                         BinCache& c) {
  if (c.bin != dg) {
    bin_cache_flush(c, cnt, mass);
    c.bin = dg;
  }
  c.cnt += 1;
  c.mass += fx_from_bits(pb, err);
}

}  // namespace sv
