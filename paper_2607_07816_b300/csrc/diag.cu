// Gates with one nonzero entry per row and column, applied term by term.
//
// Diagonal gates (CZ, RZ, phase gates and their products): Eq. (3) with
// U[r'][r] = 0 for r' != r maps every term to itself, so the grouping of
// Sec. IV-A brings nothing together and the keys do not change.
// The state stays in the order it is in (no regrouping: the stored-key order
// and the qubit order are kept), and each amplitude is multiplied in place
// by its diagonal entry, with the same fused multiply-add sequence as the
// group mat-vec for a group with one present member, so the result is the
// one the general path computes, bit for bit.  The kernel also writes each
// term's probability bits, sums the exact fixed-point total mass and counts
// exact zeros (removed by the caller with the order-preserving pass).
//
// Monomial gates (permutations with phases: X, CNOT, Toffoli, C3X): every
// term again has one output, with the gate bits r replaced by r' = pi(r).
// The regrouping sorts the terms by their output key directly (it
// partitions by pi(r) instead of r), so the merged keys are the outputs in
// the gate's order and one streaming pass multiplies each gathered amplitude
// by its entry; no group scan and no group mat-vec are needed.
#include "c64_exact.cuh"
#include "internal.h"
#include "launch.cuh"
#include "select.cuh"

namespace sv {

constexpr int DG_BLOCK = 256, DG_ITEMS = 4;

template <typename Real>
struct DCplx;
template <>
struct DCplx<double> {
  typedef double2 T;
  __device__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};
template <>
struct DCplx<float> {
  typedef float2 T;
  __device__ static float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};

// x times an entry that is +-1 or +-i, with the fused chain of the general
// path: each product is exact and the chain adds it to +0, so the result is
// a component of x, negated or not, with -0 turned into +0.  Taken with
// integer operations (the FP64 pipe is the scarce unit of the complex128
// path).
__device__ __forceinline__ double unit_part(double v, bool neg) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v) ^ ((unsigned long long)neg << 63);
  if ((b << 1) == 0ull) b = 0ull;
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ float unit_part(float v, bool neg) {
  uint32_t b = __float_as_uint(v) ^ ((uint32_t)neg << 31);
  if ((b << 1) == 0u) b = 0u;
  return __uint_as_float(b);
}

// y = u x for one entry u = (ur, ui) with nonzero components rz / iz; unit:
// u is one of +-1, +-i (neg: its nonzero component is -1).
template <typename Real>
__device__ __forceinline__ void entry_times(Real ur, Real ui, bool rz, bool iz, bool unit, bool neg, Real xr, Real xi,
                                            Real& re, Real& im) {
  re = (Real)0;
  im = (Real)0;
  if (unit) {
    if (rz) {  // u = s: (s xr, s xi)
      re = unit_part(xr, neg);
      im = unit_part(xi, neg);
    } else {  // u = s i: (-s xi, s xr)
      re = unit_part(xi, !neg);
      im = unit_part(xr, neg);
    }
    return;
  }
  if (rz) {
    re = DCplx<Real>::fma(ur, xr, re);
    im = DCplx<Real>::fma(ur, xi, im);
  }
  if (iz) {
    re = DCplx<Real>::fma(-ui, xi, re);
    im = DCplx<Real>::fma(ui, xr, im);
  }
}

template <typename Real>
__global__ void __launch_bounds__(DG_BLOCK) k_diag_apply(const uint64_t* __restrict__ keys,
                                                        typename DCplx<Real>::T* __restrict__ amps,
                                                        uint64_t* __restrict__ probs, uint64_t n,
                                                        const DiagParams dp, Ctl* ctl) {
  pdl_prologue();
  typedef typename DCplx<Real>::T C2;
  __shared__ Real s_ur[16], s_ui[16];
  if (threadIdx.x < 16) {
    s_ur[threadIdx.x] = (Real)dp.ur[threadIdx.x];  // complex64: U rounded to float, as in the mat-vec
    s_ui[threadIdx.x] = (Real)dp.ui[threadIdx.x];
  }
  __syncthreads();
  const int m = dp.m;
  u128 tot = 0;
  uint32_t zeros = 0;
  const uint64_t stride = (uint64_t)gridDim.x * DG_BLOCK * DG_ITEMS;
  for (uint64_t b = (uint64_t)blockIdx.x * DG_BLOCK * DG_ITEMS + threadIdx.x; b < n; b += stride) {
    uint64_t k[DG_ITEMS];
    C2 x[DG_ITEMS];
#pragma unroll
    for (int j = 0; j < DG_ITEMS; ++j) {  // all loads first
      const uint64_t i = b + (uint64_t)j * DG_BLOCK;
      if (i < n) {
        k[j] = keys[i];
        x[j] = amps[i];
      }
    }
#pragma unroll
    for (int j = 0; j < DG_ITEMS; ++j) {
      const uint64_t i = b + (uint64_t)j * DG_BLOCK;
      if (i >= n) continue;
      uint32_t r = 0;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t < m) r |= (uint32_t)((k[j] >> dp.qpos[t]) & 1ull) << t;
      Real re, im;
      entry_times(s_ur[r], s_ui[r], (dp.rnz >> r) & 1u, (dp.inz >> r) & 1u, (dp.unit >> r) & 1u, (dp.uneg >> r) & 1u,
                  x[j].x, x[j].y, re, im);
      C2 y;
      y.x = re;
      y.y = im;
      amps[i] = y;
      const uint64_t pb = amp_prob_bits(y);
      probs[i] = pb;
      tot += fx_from_bits(pb, &ctl->err);
      zeros += (re == (Real)0 && im == (Real)0) ? 1u : 0u;
    }
  }
  tot = warp_sum_u128(tot);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) zeros += __shfl_xor_sync(0xffffffffu, zeros, o);
  if ((threadIdx.x & 31) == 0) {
    if (tot) atomic_add_u128(&ctl->total_mass_hi, &ctl->total_mass_lo, tot);
    if (zeros) atomicAdd((unsigned long long*)&ctl->count[3], (unsigned long long)zeros);
  }
}

void launch_diag_apply(int prec, const uint64_t* keys, void* amps, uint64_t* probs, uint64_t n, const DiagParams& dp,
                       Ctl* ctl, cudaStream_t st) {
  if (n == 0) return;
  uint64_t blocks = (n + DG_BLOCK * DG_ITEMS - 1) / (DG_BLOCK * DG_ITEMS);
  if (blocks > 148ull * 8) blocks = 148ull * 8;
  if (prec == 0)
    launch_pdl(k_diag_apply<double>, (unsigned)blocks, DG_BLOCK, 0, st, keys, (double2*)amps, probs, n, dp, ctl);
  else
    launch_pdl(k_diag_apply<float>, (unsigned)blocks, DG_BLOCK, 0, st, keys, (float2*)amps, probs, n, dp, ctl);
}

template <typename Real>
__global__ void __launch_bounds__(DG_BLOCK) k_mono_apply(const uint64_t* __restrict__ sk,
                                                        const uint32_t* __restrict__ sidx, uint64_t n,
                                                        const typename DCplx<Real>::T* __restrict__ amps_in,
                                                        const MonoParams mp, uint64_t* __restrict__ keys_out,
                                                        typename DCplx<Real>::T* __restrict__ amps_out,
                                                        uint64_t* __restrict__ probs_out, Ctl* ctl) {
  pdl_prologue();
  typedef typename DCplx<Real>::T C2;
  __shared__ Real s_ur[16], s_ui[16];
  if (threadIdx.x < 16) {
    s_ur[threadIdx.x] = (Real)mp.ur[threadIdx.x];
    s_ui[threadIdx.x] = (Real)mp.ui[threadIdx.x];
  }
  __syncthreads();
  const int vb = mp.vbits;
  const uint32_t dmask = (1u << mp.m) - 1u;
  const uint64_t imask = vb ? ((1ull << vb) - 1ull) : 0ull;
  u128 tot = 0;
  uint32_t zeros = 0;
  const uint64_t stride = (uint64_t)gridDim.x * DG_BLOCK * DG_ITEMS;
  for (uint64_t b = (uint64_t)blockIdx.x * DG_BLOCK * DG_ITEMS + threadIdx.x; b < n; b += stride) {
    uint64_t v[DG_ITEMS];
    C2 x[DG_ITEMS];
#pragma unroll
    for (int j = 0; j < DG_ITEMS; ++j) {
      const uint64_t i = b + (uint64_t)j * DG_BLOCK;
      if (i < n) v[j] = sk[i];
    }
#pragma unroll
    for (int j = 0; j < DG_ITEMS; ++j) {  // the gathers, all in flight together
      const uint64_t i = b + (uint64_t)j * DG_BLOCK;
      if (i < n) x[j] = amps_in[vb ? (v[j] & imask) : (uint64_t)sidx[i]];
    }
#pragma unroll
    for (int j = 0; j < DG_ITEMS; ++j) {
      const uint64_t i = b + (uint64_t)j * DG_BLOCK;
      if (i >= n) continue;
      const uint64_t key = v[j] >> vb;  // the output's stored key: rest above, r' at the bottom
      const uint32_t ro = (uint32_t)key & dmask;
      Real re, im;
      entry_times(s_ur[ro], s_ui[ro], (mp.rnz >> ro) & 1u, (mp.inz >> ro) & 1u, (mp.unit >> ro) & 1u,
                  (mp.uneg >> ro) & 1u, x[j].x, x[j].y, re, im);
      C2 y;
      y.x = re;
      y.y = im;
      keys_out[i] = key;
      amps_out[i] = y;
      const uint64_t pb = amp_prob_bits(y);
      probs_out[i] = pb;
      tot += fx_from_bits(pb, &ctl->err);
      zeros += (re == (Real)0 && im == (Real)0) ? 1u : 0u;
    }
  }
  tot = warp_sum_u128(tot);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) zeros += __shfl_xor_sync(0xffffffffu, zeros, o);
  if ((threadIdx.x & 31) == 0) {
    if (tot) atomic_add_u128(&ctl->total_mass_hi, &ctl->total_mass_lo, tot);
    if (zeros) atomicAdd((unsigned long long*)&ctl->count[3], (unsigned long long)zeros);
  }
}

void launch_mono_apply(int prec, const uint64_t* sk, const uint32_t* sidx, uint64_t n, const void* amps_in,
                       const MonoParams& mp, uint64_t* keys_out, void* amps_out, uint64_t* probs_out, Ctl* ctl,
                       cudaStream_t st) {
  if (n == 0) return;
  uint64_t blocks = (n + DG_BLOCK * DG_ITEMS - 1) / (DG_BLOCK * DG_ITEMS);
  if (blocks > 148ull * 8) blocks = 148ull * 8;
  if (prec == 0)
    launch_pdl(k_mono_apply<double>, (unsigned)blocks, DG_BLOCK, 0, st, sk, sidx, n, (const double2*)amps_in, mp,
               keys_out, (double2*)amps_out, probs_out, ctl);
  else
    launch_pdl(k_mono_apply<float>, (unsigned)blocks, DG_BLOCK, 0, st, sk, sidx, n, (const float2*)amps_in, mp,
               keys_out, (float2*)amps_out, probs_out, ctl);
}

}  // namespace sv
