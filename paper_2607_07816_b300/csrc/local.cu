// Local gate application inside shared memory.
//
// A gate whose qubits avoid a set P of bucket qubits only combines terms that
// agree on P (partners differ only in the gate qubits, Sec. I and Sec.
// IV-A), so on a state where such buckets are contiguous, whole buckets can
// be processed independently: one block loads the buckets that start in its
// chunk of the state, sorts them in shared memory by the gate's sort key (P
// on top, the gate qubits at the bottom in local-index order), finds the
// partner groups, computes each output y[r'] = sum over present r ascending
// of U[r'][r] x[r] (Eq. 3 with the same fused multiply-add order as the rest
// of the library) and writes the outputs of the batch into one contiguous
// range.  The range is reserved with one atomic add, sized by the outputs
// that are structurally nonzero (a present input meets a nonzero entry of
// U's row); outputs that cancel exactly are written with a zero amplitude
// and counted, and a later order-preserving pass drops them.  The library
// runs it with P empty on states of at most one batch (a single launch for
// the whole gate); larger states take the sorted path, which measured as
// fast or faster on this GPU.
#include "c64_exact.cuh"
#include "internal.h"
#include "launch.cuh"
#include "tile.cuh"

namespace sv {

constexpr int LG_THREADS = 1024;
constexpr int LG_WARPS = LG_THREADS / 32;
constexpr int LG_ITEMS = LOCAL_CAP / LG_THREADS;  // 4

template <typename Real>
struct LCplx;
template <>
struct LCplx<double> {
  typedef double2 T;
};
template <>
struct LCplx<float> {
  typedef float2 T;
};

__device__ __forceinline__ double lfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float lfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <typename Real>
struct LocalSmem {
  uint64_t sk[2][LOCAL_CAP];          // sort keys (ping-pong); the idle half holds group data
  uint16_t ix[2][LOCAL_CAP];          // batch positions (ping-pong)
  uint32_t whist[LG_WARPS][RADIX];    // per-warp digit counters
  uint64_t fwd[16][16];               // key -> sort key
  uint64_t inv[16][16];               // sort key -> key
  Real U[512];
  uint32_t re_nz[16], im_nz[16], st_nz[16];
  uint32_t dsum[RADIX];
  uint32_t wtot[LG_WARPS];
  uint64_t red_or, red_and;
  uint64_t bounds[2];
  uint64_t out_base;
  uint64_t batch;
  uint32_t ngroups;
  uint32_t total;
};

// Group tables placed in the idle sort buffers once the batch is sorted:
// gstart (u16) in the idle index buffer, gmask and gout (u32) in the idle
// key buffer.
struct GroupView {
  uint16_t* gstart;  // [LOCAL_CAP] first member of each group (the batch end closes the last)
  uint32_t* gmask;   // [LOCAL_CAP] present inputs (low 16 bits), structural outputs (high 16)
  uint32_t* gout;    // [LOCAL_CAP] exclusive structural output offset per group (SC closes)
};

// Start of batch c: the first bucket boundary at or after c * LOCAL_CHUNK
// (n when none is left).  The bucket covering that position ends within
// LOCAL_BUCKET_MAX terms if buckets respect the limit; otherwise ERR_BUCKET.
// All 32 lanes of a warp call it and get the same value.
__device__ __forceinline__ uint64_t batch_start(const uint64_t* __restrict__ keys, uint64_t n,
                                                uint64_t pmask, uint64_t c, uint32_t* err) {
  const int lane = threadIdx.x & 31;
  if (c == 0) return 0;
  const uint64_t pos0 = c * (uint64_t)LOCAL_CHUNK;
  if (pos0 >= n) return n;
  const uint64_t end = n < pos0 + LOCAL_BUCKET_MAX + 1 ? n : pos0 + LOCAL_BUCKET_MAX + 1;
  for (uint64_t b = pos0; b < end; b += 32) {
    const uint64_t i = b + lane;
    const bool f = i < end && ((keys[i] ^ keys[i - 1]) & pmask) != 0;
    const uint32_t bal = __ballot_sync(0xffffffffu, f);
    if (bal) return b + (uint64_t)(__ffs(bal) - 1);
  }
  if (end == n) return n;
  if (lane == 0) atomicOr(err, ERR_BUCKET);
  return end;
}

// Exclusive scan of one value per thread over the block.
__device__ __forceinline__ uint32_t lg_block_scan(uint32_t v, uint32_t* wtot, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtot[warp] = x;
  __syncthreads();
  uint32_t base = 0, all = 0;
  for (int w = 0; w < LG_WARPS; ++w) {
    if (w < warp) base += wtot[w];
    all += wtot[w];
  }
  __syncthreads();
  if (total) *total = all;
  return base + x - v;
}

// One stable LSD pass over the batch on the 8-bit digit at `shift`.
template <typename Real>
__device__ __forceinline__ void lg_sort_pass(LocalSmem<Real>& sm, int from, uint32_t B, int shift) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  for (int i = lane; i < RADIX; i += 32) sm.whist[warp][i] = 0;
  __syncwarp();
  uint64_t k[LG_ITEMS];
  uint16_t v[LG_ITEMS];
  uint32_t dg[LG_ITEMS], rk[LG_ITEMS];
#pragma unroll
  for (int j = 0; j < LG_ITEMS; ++j) {
    const uint32_t i = (uint32_t)warp * 32 * LG_ITEMS + j * 32 + lane;
    const bool valid = i < B;
    k[j] = valid ? sm.sk[from][i] : 0ull;
    v[j] = valid ? sm.ix[from][i] : (uint16_t)0;
    dg[j] = valid ? (uint32_t)((k[j] >> shift) & (RADIX - 1)) : (uint32_t)RADIX;
  }
#pragma unroll
  for (int j = 0; j < LG_ITEMS; ++j) {
    const uint32_t peers = __match_any_sync(0xffffffffu, dg[j]);
    const int leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if (lane == leader && dg[j] < RADIX) {
      old = sm.whist[warp][dg[j]];
      sm.whist[warp][dg[j]] = old + __popc(peers);
    }
    rk[j] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
    __syncwarp();
  }
  __syncthreads();
  uint32_t tot = 0;
  if (threadIdx.x < RADIX) {
    for (int w = 0; w < LG_WARPS; ++w) {
      const uint32_t c = sm.whist[w][threadIdx.x];
      sm.whist[w][threadIdx.x] = tot;
      tot += c;
    }
  }
  const uint32_t off = lg_block_scan(threadIdx.x < RADIX ? tot : 0u, sm.wtot, nullptr);
  if (threadIdx.x < RADIX) sm.dsum[threadIdx.x] = off;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < LG_ITEMS; ++j) {
    if (dg[j] < RADIX) {
      const uint32_t pos = sm.dsum[dg[j]] + sm.whist[warp][dg[j]] + rk[j];
      sm.sk[from ^ 1][pos] = k[j];
      sm.ix[from ^ 1][pos] = v[j];
    }
  }
  __syncthreads();
}

template <typename Real>
__global__ void __launch_bounds__(LG_THREADS, 1) k_local_gate(
    const uint64_t* __restrict__ keys, const typename LCplx<Real>::T* __restrict__ amps, uint64_t n,
    const GateParams gp, uint64_t* __restrict__ keys_out, typename LCplx<Real>::T* __restrict__ amps_out,
    uint64_t* __restrict__ probs_out, Ctl* ctl) {
  typedef typename LCplx<Real>::T C2;
  extern __shared__ __align__(16) uint8_t s_dyn[];
  LocalSmem<Real>& sm = *reinterpret_cast<LocalSmem<Real>*>(s_dyn);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = gp.m, d = 1 << m;
  const uint32_t dmask = (uint32_t)d - 1u;
  const int top_shift = gp.n - gp.tbits;  // bucket bits sit above this
  for (int i = tid; i < 256; i += LG_THREADS) {
    (&sm.fwd[0][0])[i] = (&gp.perm->fwd[0][0])[i];
    (&sm.inv[0][0])[i] = (&gp.perm->inv[0][0])[i];
  }
  for (int i = tid; i < 2 * d * d; i += LG_THREADS) sm.U[i] = (Real)gp.U[i];
  if (tid < 16) {
    sm.re_nz[tid] = gp.re_nz[tid];
    sm.im_nz[tid] = gp.im_nz[tid];
    sm.st_nz[tid] = gp.re_nz[tid] | gp.im_nz[tid];
  }
  const uint64_t nbatches = (n + LOCAL_CHUNK - 1) / LOCAL_CHUNK;
  uint64_t max_bucket = 0;
  while (true) {
    if (tid == 0) {
      sm.batch = atomicAdd((unsigned long long*)&ctl->tile_counter[3], 1ull);
      sm.red_or = 0;
      sm.red_and = ~0ull;
    }
    __syncthreads();
    const uint64_t c = sm.batch;
    if (c >= nbatches) break;
    if (warp < 2) {
      const uint64_t b = batch_start(keys, n, gp.pmask, c + warp, &ctl->err);
      if (lane == 0) sm.bounds[warp] = b;
    }
    __syncthreads();
    const uint64_t s = sm.bounds[0], e = sm.bounds[1];
    uint32_t B = e > s ? (uint32_t)(e - s) : 0u;
    if (e > s && e - s > (uint64_t)LOCAL_CAP) {
      if (tid == 0) atomicOr(&ctl->err, ERR_BUCKET);
      B = 0;
    }
    if (B == 0) {
      __syncthreads();
      continue;
    }
    // ---- load and permute the batch
    uint64_t orv = 0, andv = ~0ull;
    for (uint32_t i = tid; i < B; i += LG_THREADS) {
      const uint64_t x = permute_bits(sm.fwd, keys[s + i]);
      sm.sk[0][i] = x;
      sm.ix[0][i] = (uint16_t)i;
      orv |= x;
      andv &= x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      orv |= __shfl_xor_sync(0xffffffffu, (unsigned long long)orv, o);
      andv &= __shfl_xor_sync(0xffffffffu, (unsigned long long)andv, o);
    }
    if (lane == 0) {
      atomicOr((unsigned long long*)&sm.red_or, (unsigned long long)orv);
      atomicAnd((unsigned long long*)&sm.red_and, (unsigned long long)andv);
    }
    __syncthreads();
    // ---- sort by the sort key, only on digits that vary inside the batch
    const uint64_t diff = sm.red_or ^ sm.red_and;
    int cur = 0;
    for (int shift = 0; shift < gp.n; shift += RADIX_BITS) {
      if (((diff >> shift) & (RADIX - 1)) == 0) continue;
      lg_sort_pass(sm, cur, B, shift);
      cur ^= 1;
    }
    // ---- partner groups
    GroupView gv;
    gv.gmask = reinterpret_cast<uint32_t*>(sm.sk[cur ^ 1]);
    gv.gout = gv.gmask + LOCAL_CAP;   // the idle key buffer holds 2 * LOCAL_CAP u32
    gv.gstart = sm.ix[cur ^ 1];       // LOCAL_CAP u16: the terminator is kept in ngroups/total
    uint32_t run = 0;
    uint32_t gpos[LG_ITEMS];
    bool gflag[LG_ITEMS];
#pragma unroll
    for (int j = 0; j < LG_ITEMS; ++j) {
      const uint32_t i = (uint32_t)warp * 32 * LG_ITEMS + j * 32 + lane;
      gflag[j] = i < B && (i == 0 || (sm.sk[cur][i] >> m) != (sm.sk[cur][i - 1] >> m));
      const uint32_t bal = __ballot_sync(0xffffffffu, gflag[j]);
      gpos[j] = run + __popc(bal & ((1u << lane) - 1u));
      run += __popc(bal);
    }
    uint32_t G = 0;
    const uint32_t wbase = lg_block_scan(lane == 31 ? run : 0u, sm.wtot, &G);
    const uint32_t wofs = __shfl_sync(0xffffffffu, wbase, 31);
#pragma unroll
    for (int j = 0; j < LG_ITEMS; ++j) {
      if (gflag[j]) gv.gstart[wofs + gpos[j]] = (uint16_t)((uint32_t)warp * 32 * LG_ITEMS + j * 32 + lane);
    }
    if (tid == 0) sm.ngroups = G;
    __syncthreads();
    // ---- present inputs and structurally nonzero outputs of each group
    const uint32_t per = (G + LG_THREADS - 1) / LG_THREADS;
    const uint32_t ga = tid * per, gb = min(G, ga + per);
    uint32_t cnt = 0;
    for (uint32_t g = ga; g < gb; ++g) {
      uint32_t pm = 0;
      const uint32_t qe = g + 1 < G ? gv.gstart[g + 1] : B;
      for (uint32_t q = gv.gstart[g]; q < qe; ++q) pm |= 1u << (uint32_t)(sm.sk[cur][q] & dmask);
      uint32_t om = 0;
      for (int r = 0; r < d; ++r)
        if (sm.st_nz[r] & pm) om |= 1u << r;
      gv.gmask[g] = pm | (om << 16);
      gv.gout[g] = __popc(om);
      cnt += __popc(om);
    }
    uint32_t SC = 0;
    uint32_t off = lg_block_scan(cnt, sm.wtot, &SC);
    for (uint32_t g = ga; g < gb; ++g) {
      const uint32_t v = gv.gout[g];
      gv.gout[g] = off;
      off += v;
    }
    if (tid == 0) {
      sm.out_base = SC ? atomicAdd((unsigned long long*)&ctl->count[1], (unsigned long long)SC) : 0ull;
    }
    __syncthreads();
    // largest output bucket of the batch (buckets are whole inside a batch)
    if (gp.tbits > 0) {
      for (uint32_t g = tid; g < G; g += LG_THREADS) {
        const uint64_t bk = sm.sk[cur][gv.gstart[g]] >> top_shift;
        if (g == 0 || (sm.sk[cur][gv.gstart[g - 1]] >> top_shift) != bk) {
          uint32_t j = g + 1;
          while (j < G && (sm.sk[cur][gv.gstart[j]] >> top_shift) == bk) ++j;
          const uint64_t size = (j < G ? gv.gout[j] : SC) - gv.gout[g];
          max_bucket = size > max_bucket ? size : max_bucket;
        }
      }
    } else if (tid == 0) {
      max_bucket = SC > max_bucket ? SC : max_bucket;
    }
    // ---- outputs
    const uint64_t obase = sm.out_base;
    uint32_t zeros = 0;
    for (uint32_t ls = tid; ls < (G << m); ls += LG_THREADS) {
      const uint32_t g = ls >> m, ro = ls & dmask;
      const uint32_t gm = gv.gmask[g];
      const uint32_t pm = gm & 0xffffu, om = gm >> 16;
      if (!((om >> ro) & 1u)) continue;
      const uint32_t h = gv.gstart[g];
      const uint32_t rnz = sm.re_nz[ro] & pm, inz = sm.im_nz[ro] & pm;
      uint32_t cols = rnz | inz;
      Real re = (Real)0, im = (Real)0;
      while (cols) {
        const int r = __ffs(cols) - 1;
        cols &= cols - 1u;
        const C2 x = amps[s + sm.ix[cur][h + __popc(pm & ((1u << r) - 1u))]];
        const Real ur = sm.U[2 * (ro * d + r)], ui = sm.U[2 * (ro * d + r) + 1];
        if ((rnz >> r) & 1u) {
          re = lfma(ur, x.x, re);
          im = lfma(ur, x.y, im);
        }
        if ((inz >> r) & 1u) {
          re = lfma(-ui, x.y, re);
          im = lfma(ui, x.x, im);
        }
      }
      const uint64_t o = obase + gv.gout[g] + __popc(om & ((1u << ro) - 1u));
      keys_out[o] = permute_bits(sm.inv, ((sm.sk[cur][h] >> m) << m) | ro);
      C2 yv;
      yv.x = re;
      yv.y = im;
      amps_out[o] = yv;
      probs_out[o] = amp_prob_bits(re, im);
      if (re == (Real)0 && im == (Real)0) ++zeros;
    }
    if (zeros) atomicAdd((unsigned long long*)&ctl->count[3], (unsigned long long)zeros);
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t y = __shfl_xor_sync(0xffffffffu, (unsigned long long)max_bucket, o);
    max_bucket = y > max_bucket ? y : max_bucket;
  }
  if (lane == 0 && max_bucket) atomicMax((unsigned long long*)&ctl->count[0], (unsigned long long)max_bucket);
}

cudaError_t local_prepare() {
  static DeviceOnce once;
  return once.run([] {
    cudaError_t e = cudaFuncSetAttribute(k_local_gate<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(LocalSmem<double>));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_local_gate<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sizeof(LocalSmem<float>));
    return e;
  });
}

void launch_local_gate(int prec, const uint64_t* keys, const void* amps, uint64_t n, const GateParams& gp,
                       uint64_t* keys_out, void* amps_out, uint64_t* probs_out, Ctl* ctl, cudaStream_t st) {
  (void)local_prepare();  // checked at the handle's creation; a launch without it fails loudly
  cudaMemsetAsync(&ctl->tile_counter[3], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[0], 0, sizeof(uint64_t) * 2, st);  // largest bucket, output count
  cudaMemsetAsync(&ctl->count[3], 0, sizeof(uint64_t), st);       // exact zeros
  if (n == 0) return;
  const uint64_t nb = (n + LOCAL_CHUNK - 1) / LOCAL_CHUNK;
  const uint64_t grid = nb < 148 ? nb : 148;
  if (prec == 0)
    k_local_gate<double><<<(unsigned)grid, LG_THREADS, sizeof(LocalSmem<double>), st>>>(
        keys, (const double2*)amps, n, gp, keys_out, (double2*)amps_out, probs_out, ctl);
  else
    k_local_gate<float><<<(unsigned)grid, LG_THREADS, sizeof(LocalSmem<float>), st>>>(
        keys, (const float2*)amps, n, gp, keys_out, (float2*)amps_out, probs_out, ctl);
}

// ---------------------------------------------------------------- zero removal
constexpr int DZ_BLOCK = 256, DZ_ITEMS = 8;

template <typename C2>
__global__ void __launch_bounds__(DZ_BLOCK) k_drop_zero_terms(
    const uint64_t* __restrict__ keys, const C2* __restrict__ amps, const uint64_t* __restrict__ probs,
    uint64_t n, uint64_t* __restrict__ keys_out, C2* __restrict__ amps_out, uint64_t* __restrict__ probs_out,
    uint64_t* lookback, Ctl* ctl) {
  typedef TileLayout<DZ_BLOCK, DZ_ITEMS> L;
  __shared__ CompactShared<DZ_BLOCK> cs;
  __shared__ uint64_t s_tile;
  const uint64_t tiles = (n + L::TILE - 1) / L::TILE;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd((unsigned long long*)&ctl->tile_counter[2], 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= tiles) break;
    const uint64_t base = tile * L::TILE;
    bool flag[DZ_ITEMS];
    uint32_t pos[DZ_ITEMS];
    C2 a[DZ_ITEMS];
#pragma unroll
    for (int j = 0; j < DZ_ITEMS; ++j) {
      const uint64_t i = L::index(base, j);
      flag[j] = false;
      if (i < n) {
        a[j] = amps[i];
        flag[j] = !(a[j].x == 0 && a[j].y == 0);
      }
    }
    tile_compact<DZ_BLOCK, DZ_ITEMS>(flag, pos, cs, lookback, tile, &ctl->err);
#pragma unroll
    for (int j = 0; j < DZ_ITEMS; ++j) {
      if (flag[j]) {
        const uint64_t i = L::index(base, j);
        const uint64_t o = cs.tile_base_out + pos[j];
        keys_out[o] = keys[i];
        amps_out[o] = a[j];
        probs_out[o] = probs[i];
      }
    }
    if (tile == tiles - 1 && threadIdx.x == 0) ctl->count[2] = cs.tile_base_out + cs.tile_total;
    __syncthreads();
  }
}

void launch_drop_zero_terms(int prec, const uint64_t* keys, const void* amps, const uint64_t* probs,
                            uint64_t n, uint64_t* keys_out, void* amps_out, uint64_t* probs_out,
                            uint64_t* lookback, Ctl* ctl, cudaStream_t st) {
  const uint64_t tiles = (n + DZ_BLOCK * DZ_ITEMS - 1) / (DZ_BLOCK * DZ_ITEMS);
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * (tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[2], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[2], 0, sizeof(uint64_t), st);
  if (n == 0) return;
  const uint64_t grid = tiles < 148 * 8 ? tiles : 148 * 8;
  if (prec == 0)
    k_drop_zero_terms<double2><<<(unsigned)grid, DZ_BLOCK, 0, st>>>(
        keys, (const double2*)amps, probs, n, keys_out, (double2*)amps_out, probs_out, lookback, ctl);
  else
    k_drop_zero_terms<float2><<<(unsigned)grid, DZ_BLOCK, 0, st>>>(
        keys, (const float2*)amps, probs, n, keys_out, (float2*)amps_out, probs_out, lookback, ctl);
}

}  // namespace sv
