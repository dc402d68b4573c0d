// Gate application helpers for the radix-sort grouping and the expand-first
// form: the key transform with digit histograms and the partner-group heads.
//
// Sec. IV-A: every amplitude meets the column of U selected by its bits on
// the gate qubits; all amplitudes whose basis states agree outside those bits
// form one group, whose 2^m outputs are y[r'] = sum_r U[r'][r] x[r] (Eq. 3
// generalised).  The group is made contiguous by sorting on the key with the
// gate bits moved to the bottom, so a group is a run of equal sk >> m with its
// members in ascending r.
#include "c64_exact.cuh"
#include "internal.h"
#include "launch.cuh"
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

// ------------------------------------------------------------------ gate tables
constexpr uint32_t RESET_PER_BLOCK = 256 * 16;

__global__ void __launch_bounds__(256) k_store_tables(const GateTables t, GateTables* __restrict__ dst,
                                                      uint32_t words, const GateReset r) {
  pdl_prologue();
  if (blockIdx.x == 0) {
    const uint64_t* src = reinterpret_cast<const uint64_t*>(&t);
    uint64_t* out = reinterpret_cast<uint64_t*>(dst);
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) out[i] = src[i];
  }
  if (!r.ctl) return;
  if (blockIdx.x == 0 && threadIdx.x < 16) r.part_hist[threadIdx.x] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    r.ctl->tile_counter[0] = 0;
    r.ctl->tile_counter[1] = 0;
    for (int i = 0; i < 4; ++i) r.ctl->count[i] = 0;
    r.ctl->total_mass_hi = r.ctl->total_mass_lo = 0;
  }
  const uint32_t e = blockIdx.x * RESET_PER_BLOCK + threadIdx.x;
  for (uint32_t i = e; i < r.lb_words && i < (blockIdx.x + 1) * RESET_PER_BLOCK; i += blockDim.x) r.lb[i] = 0;
}

void launch_store_tables(const GateTables& t, GateTables* dst, size_t bytes, const GateReset& r, cudaStream_t st) {
  const uint32_t blocks = r.ctl ? 1u + r.lb_words / RESET_PER_BLOCK : 1u;
  launch_pdl(k_store_tables, blocks, 256, 0, st, t, dst, (uint32_t)((bytes + 7) / 8), r);
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

}  // namespace sv
