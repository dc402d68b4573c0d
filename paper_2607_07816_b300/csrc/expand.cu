// Expand-first gate application: the paper's own formulation (Sec. IV-A).
//
// Every amplitude is multiplied by the column of U its gate bits select, so
// each term contributes to the 2^m basis states that differ from it in the
// gate qubits; contributions to the same basis state are then summed (a
// segmented sum).  Here each contribution is a record (sort key, source
// term): the sort key is the output's sort key (bits outside the gate, then
// the output's gate bits r') followed by the source's gate bits r, so after
// one radix sort the contributions to an output are contiguous and in
// ascending r.  The reduction then runs, per output, the same fused
// multiply-add chain as the group-first path (present inputs in ascending r,
// zero U components skipped), so both forms give the same bits; the outputs
// come out in the same order as well (ascending output sort key).  This form
// sorts 2^m times as many records as the group-first path, which sorts the
// terms once and expands inside the mat-vec.
#include "c64_exact.cuh"
#include "internal.h"
#include "tile.cuh"

namespace sv {

// Records i * 2^m + r' for every term i and output r' (the permutation moves
// the gate bits of the key to the bottom, so s = rest << m | r).
__global__ void __launch_bounds__(256) k_expand_records(const uint64_t* __restrict__ keys, uint64_t n,
                                                        const BitPerm* __restrict__ perm, int m,
                                                        uint64_t* __restrict__ sk, uint32_t* __restrict__ sidx,
                                                        uint32_t* __restrict__ hist, int passes) {
  __shared__ uint32_t sh[MAX_PASSES][RADIX];
  __shared__ uint64_t fwd[16][16];
  for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) (&sh[0][0])[i] = 0;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) (&fwd[0][0])[i] = (&perm->fwd[0][0])[i];
  __syncthreads();
  const uint32_t d = 1u << m;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = permute_bits(fwd, keys[i]);
    const uint64_t rest = s >> m, r = s & (d - 1);
    for (uint32_t ro = 0; ro < d; ++ro) {
      const uint64_t rec = (((rest << m) | ro) << m) | r;
      sk[i * d + ro] = rec;
      sidx[i * d + ro] = (uint32_t)i;
      for (int p = 0; p < passes; ++p) atomicAdd(&sh[p][(rec >> (RADIX_BITS * p)) & (RADIX - 1)], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) {
    const uint32_t c = (&sh[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
}

void launch_expand_records(const uint64_t* keys, uint64_t n, const GateParams& gp, uint64_t* sk, uint32_t* sidx,
                           uint32_t* hist, int passes, cudaStream_t st) {
  cudaMemsetAsync(hist, 0, sizeof(uint32_t) * MAX_PASSES * RADIX, st);
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_expand_records<<<(unsigned)blocks, 256, 0, st>>>(keys, n, gp.perm, gp.m, sk, sidx, hist, passes);
}

template <typename Real>
struct ECplx;
template <>
struct ECplx<double> {
  typedef double2 T;
};
template <>
struct ECplx<float> {
  typedef float2 T;
};
__device__ __forceinline__ double efma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float efma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

constexpr int SR_BLOCK = 256, SR_ITEMS = 4;

// One output per segment of equal output sort key: the chain over its
// records (ascending source r); zero sums are dropped and the survivors
// compacted in segment order.
template <typename Real>
__global__ void __launch_bounds__(SR_BLOCK) k_segment_reduce(
    const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sidx, uint64_t nrec,
    const uint32_t* __restrict__ heads, const typename ECplx<Real>::T* __restrict__ amps_in, const GateParams gp,
    uint64_t* __restrict__ keys_out, typename ECplx<Real>::T* __restrict__ amps_out,
    uint64_t* __restrict__ probs_out, uint64_t* lookback, Ctl* ctl) {
  typedef TileLayout<SR_BLOCK, SR_ITEMS> L;
  typedef typename ECplx<Real>::T C2;
  __shared__ CompactShared<SR_BLOCK> cs;
  __shared__ uint64_t s_tile;
  __shared__ uint64_t s_inv[16][16];
  __shared__ Real sU[512];
  const int m = gp.m, d = 1 << m;
  for (int i = threadIdx.x; i < 256; i += SR_BLOCK) (&s_inv[0][0])[i] = (&gp.perm->inv[0][0])[i];
  for (int i = threadIdx.x; i < 2 * d * d; i += SR_BLOCK) sU[i] = (Real)gp.U[i];
  __syncthreads();
  const uint64_t G = ctl->count[0];
  const uint64_t tiles = (G + L::TILE - 1) / L::TILE;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd((unsigned long long*)&ctl->tile_counter[1], 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= tiles) break;
    const uint64_t base = tile * L::TILE;
    bool flag[SR_ITEMS];
    uint32_t pos[SR_ITEMS];
    Real yr[SR_ITEMS], yi[SR_ITEMS];
    uint64_t ykey[SR_ITEMS];
#pragma unroll
    for (int j = 0; j < SR_ITEMS; ++j) {
      const uint64_t g = L::index(base, j);
      Real re = (Real)0, im = (Real)0;
      bool f = false;
      uint64_t key = 0;
      if (g < G) {
        const uint64_t h = heads[g];
        const uint64_t e = g + 1 < G ? (uint64_t)heads[g + 1] : nrec;
        const uint64_t os = sk[h] >> m;  // output sort key: rest << m | r'
        const uint32_t ro = (uint32_t)(os & (uint64_t)(d - 1));
        const uint32_t rnz_all = gp.re_nz[ro], inz_all = gp.im_nz[ro];
        for (uint64_t i = h; i < e; ++i) {
          const uint32_t r = (uint32_t)(sk[i] & (uint64_t)(d - 1));
          const bool rnz = (rnz_all >> r) & 1u, inz = (inz_all >> r) & 1u;
          if (!rnz && !inz) continue;
          const C2 x = amps_in[sidx[i]];
          const Real ur = sU[2 * (ro * d + r)], ui = sU[2 * (ro * d + r) + 1];
          if (rnz) {
            re = efma(ur, x.x, re);
            im = efma(ur, x.y, im);
          }
          if (inz) {
            re = efma(-ui, x.y, re);
            im = efma(ui, x.x, im);
          }
        }
        key = permute_bits(s_inv, os);
        f = !(re == (Real)0 && im == (Real)0);
      }
      yr[j] = re;
      yi[j] = im;
      ykey[j] = key;
      flag[j] = f;
    }
    tile_compact<SR_BLOCK, SR_ITEMS>(flag, pos, cs, lookback, tile, &ctl->err);
#pragma unroll
    for (int j = 0; j < SR_ITEMS; ++j) {
      if (flag[j]) {
        const uint64_t o = cs.tile_base_out + pos[j];
        keys_out[o] = ykey[j];
        C2 y;
        y.x = yr[j];
        y.y = yi[j];
        amps_out[o] = y;
        probs_out[o] = amp_prob_bits(y);
      }
    }
    if (tile == tiles - 1 && threadIdx.x == 0) ctl->count[1] = cs.tile_base_out + cs.tile_total;
    __syncthreads();
  }
}

void launch_segment_reduce(int prec, const uint64_t* sk, const uint32_t* sidx, uint64_t nrec, const uint32_t* heads,
                           const void* amps_in, const GateParams& gp, uint64_t* keys_out, void* amps_out,
                           uint64_t* probs_out, uint64_t* lookback, Ctl* ctl, uint64_t max_tiles, cudaStream_t st) {
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * (max_tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[1], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[1], 0, sizeof(uint64_t), st);
  if (nrec == 0) return;
  const uint64_t grid = max_tiles < 148 * 8 ? (max_tiles ? max_tiles : 1) : 148 * 8;
  if (prec == 0)
    k_segment_reduce<double><<<(unsigned)grid, SR_BLOCK, 0, st>>>(sk, sidx, nrec, heads, (const double2*)amps_in, gp,
                                                                  keys_out, (double2*)amps_out, probs_out, lookback,
                                                                  ctl);
  else
    k_segment_reduce<float><<<(unsigned)grid, SR_BLOCK, 0, st>>>(sk, sidx, nrec, heads, (const float2*)amps_in, gp,
                                                                 keys_out, (float2*)amps_out, probs_out, lookback,
                                                                 ctl);
}

}  // namespace sv
