// Gate application with output positions fixed before the arithmetic.
//
// The mat-vec of Sec. IV-A (Eq. 3) produces, per partner group, the outputs
// y[r'] = sum over present r of U[r'][r] x[r]; an output can only be nonzero
// when some present member r meets a nonzero entry U[r'][r].  Those
// structurally nonzero outputs are known from the group's members and U's
// zero pattern alone, so their positions in the candidate list -- groups in
// sort-key order, outputs in ascending r' -- are a scan that can be taken
// before any amplitude is touched:
//
//   * k_group_scan: a block stages 8192 grouped sort keys in shared memory;
//     each thread walks 32 consecutive ones, marking group heads and, per
//     head, the present mask pm (bit r: member with gate bits r present) and
//     the output mask om (bit r': some present r has U[r'][r] != 0).  The
//     head count and popc(om) are scanned over the block and over the tiles
//     (two decoupled look-backs, one warp each), and every group's head
//     position, masks and first output position are written;
//   * k_gate_apply_slots: a warp takes 32 groups, stages their members'
//     amplitudes in shared memory, orders the groups' output slots by member
//     count (so the lanes of a round run chains of equal length), and each
//     lane computes one output with the fused multiply-add chain of the rest
//     of the library (present r ascending, zero components of U skipped) and
//     writes it at its position.  No barrier or look-back follows the
//     arithmetic, so warps never wait on one another.
//
// Outputs that cancel exactly are written with a zero amplitude and counted
// in ctl->count[3]; the caller then removes them with an order-preserving
// pass, which gives the same list as dropping them here (A4 zero-drop).
#include "c64_exact.cuh"
#include "internal.h"
#include "tile.cuh"

namespace sv {

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
__device__ __forceinline__ bool is_zero_amp(double re, double im) {
  return ((__double_as_longlong(re) | __double_as_longlong(im)) << 1) == 0;
}
__device__ __forceinline__ bool is_zero_amp(float re, float im) {
  return ((__float_as_uint(re) | __float_as_uint(im)) << 1) == 0;
}

constexpr int GS_BLOCK = 512, GS_WARPS = GS_BLOCK / 32, GS_ITEMS = 16;
constexpr int GS_TILE = GS_BLOCK * GS_ITEMS;  // 8192 terms; warp w owns [512 w, 512 (w + 1))
constexpr int GS_HALO = 16;                   // a group reaches at most 15 terms past its head
constexpr size_t GS_SMEM = sizeof(uint64_t) * (GS_TILE + GS_HALO + 1);

// Term e of the staged tile (e = -1: the term before the tile) is s_k[e + 1].
// Item j of a warp's lane l is term 512 w + 32 j + l, so the lanes of an
// item hold consecutive terms and consecutive heads get consecutive group
// indices (coalesced writes).
__device__ __forceinline__ bool gs_head(const uint64_t* s_k, int e, int staged, int shift, int vb, uint32_t dmask,
                                        const uint32_t* colnz, uint32_t& pm, uint32_t& om) {
  const uint64_t gk = s_k[e + 1] >> shift;
  pm = 0;
  om = 0;
  if ((s_k[e] >> shift) == gk) return false;
  for (int t = 0; t <= (int)dmask && e + t < staged; ++t) {
    const uint64_t v = s_k[e + t + 1];
    if ((v >> shift) != gk) break;
    const uint32_t r = (uint32_t)(v >> vb) & dmask;
    pm |= 1u << r;
    om |= colnz[r];
  }
  return true;
}

__global__ void __launch_bounds__(GS_BLOCK) k_group_scan(const uint64_t* __restrict__ sk, uint64_t n,
                                                         const GateParams gp, uint32_t* __restrict__ heads,
                                                         uint32_t* __restrict__ gmask, uint64_t* __restrict__ ooff,
                                                         uint64_t* lb_heads, uint64_t* lb_out, Ctl* ctl) {
  extern __shared__ __align__(16) uint8_t s_dyn[];
  uint64_t* s_k = reinterpret_cast<uint64_t*>(s_dyn);
  __shared__ uint32_t s_wh[GS_WARPS], s_wo[GS_WARPS], s_colnz[16];
  __shared__ uint64_t s_tile, s_hbase, s_obase, s_th, s_to;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = gp.m, vb = gp.vbits, shift = m + vb;
  const uint32_t dmask = (1u << m) - 1u, lt = (1u << lane) - 1u;
  if (tid < 16) {  // colnz[r]: outputs r' with U[r'][r] != 0
    uint32_t c = 0;
    for (int ro = 0; ro < (1 << m); ++ro)
      if (((gp.re_nz[ro] | gp.im_nz[ro]) >> tid) & 1u) c |= 1u << ro;
    s_colnz[tid] = c;
  }
  const uint64_t tiles = (n + GS_TILE - 1) / GS_TILE;
  while (true) {
    if (tid == 0) s_tile = atomicAdd((unsigned long long*)&ctl->tile_counter[0], 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= tiles) break;
    const uint64_t base = tile * GS_TILE;
    const int tn = (int)(n - base < (uint64_t)GS_TILE ? n - base : (uint64_t)GS_TILE);
    const int staged = (int)(n - base < (uint64_t)(GS_TILE + GS_HALO) ? n - base : (uint64_t)(GS_TILE + GS_HALO));
    // the key before the tile must differ from the first key's group when there is none
    if (tid == 0) s_k[0] = base > 0 ? sk[base - 1] : ~sk[0];
    for (int e = tid; e < staged; e += GS_BLOCK) s_k[e + 1] = sk[base + e];
    __syncthreads();
    const int wbase = warp * 32 * GS_ITEMS;
    // pass 1: the warp's head and output counts
    uint32_t nh = 0, no = 0;
#pragma unroll 4
    for (int j = 0; j < GS_ITEMS; ++j) {
      const int e = wbase + j * 32 + lane;
      uint32_t pm, om;
      const bool f = e < tn && gs_head(s_k, e, staged, shift, vb, dmask, s_colnz, pm, om);
      nh += (uint32_t)__popc(__ballot_sync(0xffffffffu, f));
      no += __reduce_add_sync(0xffffffffu, f ? (uint32_t)__popc(om) : 0u);
    }
    if (lane == 0) {
      s_wh[warp] = nh;
      s_wo[warp] = no;
    }
    __syncthreads();
    if (warp < 2) {  // warp 0: groups, warp 1: outputs; exclusive over the warps, then over the tiles
      uint32_t* w = warp == 0 ? s_wh : s_wo;
      const uint32_t v = lane < GS_WARPS ? w[lane] : 0u;
      uint32_t x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
      const uint64_t b = lookback_exclusive_warp(warp == 0 ? lb_heads : lb_out, tile, total, &ctl->err);
      __syncwarp();
      if (lane < GS_WARPS) w[lane] = x - v;
      if (lane == 0) {
        if (warp == 0) {
          s_hbase = b;
          s_th = total;
        } else {
          s_obase = b;
          s_to = total;
        }
      }
    }
    __syncthreads();
    // pass 2: positions and coalesced writes
    uint64_t g = s_hbase + s_wh[warp], o = s_obase + s_wo[warp];
#pragma unroll 4
    for (int j = 0; j < GS_ITEMS; ++j) {
      const int e = wbase + j * 32 + lane;
      uint32_t pm = 0, om = 0;
      const bool f = e < tn && gs_head(s_k, e, staged, shift, vb, dmask, s_colnz, pm, om);
      const uint32_t hb = __ballot_sync(0xffffffffu, f);
      const uint32_t c = f ? (uint32_t)__popc(om) : 0u;
      uint32_t cx = c;
#pragma unroll
      for (int k = 1; k < 32; k <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, cx, k);
        if (lane >= k) cx += y;
      }
      if (f) {
        const uint64_t gi = g + (uint64_t)__popc(hb & lt);
        heads[gi] = (uint32_t)(base + e);
        gmask[gi] = pm | (om << 16);
        ooff[gi] = o + (cx - c);
      }
      g += (uint64_t)__popc(hb);
      o += __shfl_sync(0xffffffffu, cx, 31);
    }
    if (tile == tiles - 1 && tid == 0) {
      ctl->count[0] = s_hbase + s_th;
      ctl->count[1] = s_obase + s_to;
    }
    __syncthreads();
  }
}

void launch_group_scan(const uint64_t* sk, uint64_t n, const GateParams& gp, uint32_t* heads, uint32_t* gmask,
                       uint64_t* ooff, uint64_t* lookback, Ctl* ctl, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_group_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GS_SMEM);
    attr_set = true;
  }
  const uint64_t tiles = (n + GS_TILE - 1) / GS_TILE;
  cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * 2 * (tiles + 1), st);
  cudaMemsetAsync(&ctl->tile_counter[0], 0, sizeof(uint64_t), st);
  cudaMemsetAsync(&ctl->count[0], 0, sizeof(uint64_t) * 2, st);
  if (n == 0) return;
  const uint64_t grid = tiles < 148 * 3 ? tiles : 148 * 3;
  k_group_scan<<<(unsigned)grid, GS_BLOCK, GS_SMEM, st>>>(sk, n, gp, heads, gmask, ooff, lookback,
                                                           lookback + tiles + 1, ctl);
}

constexpr int AS_BLOCK = 256, AS_WARPS = AS_BLOCK / 32;

template <typename Real>
static size_t slots_smem(int m) {
  return (size_t)AS_WARPS * (32u << m) * (sizeof(typename SCplx<Real>::T) + sizeof(uint16_t));
}

template <typename Real>
__global__ void __launch_bounds__(AS_BLOCK) k_gate_apply_slots(
    const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sidx, const uint32_t* __restrict__ heads,
    const uint32_t* __restrict__ gmask, const uint64_t* __restrict__ ooff,
    const typename SCplx<Real>::T* __restrict__ amps_in, const GateParams gp, uint64_t* __restrict__ keys_out,
    typename SCplx<Real>::T* __restrict__ amps_out, uint64_t* __restrict__ probs_out, Ctl* ctl) {
  typedef typename SCplx<Real>::T C2;
  extern __shared__ __align__(16) uint8_t s_dyn[];
  __shared__ Real sU[512];
  __shared__ uint32_t s_re_nz[16], s_im_nz[16];
  __shared__ uint64_t s_inv[16][16];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = gp.m, d = 1 << m, vb = gp.vbits;
  const uint32_t cap = 32u << m;  // members (and output slots) of 32 groups at most
  C2* xs = reinterpret_cast<C2*>(s_dyn) + (size_t)warp * cap;
  uint16_t* slots = reinterpret_cast<uint16_t*>(reinterpret_cast<C2*>(s_dyn) + (size_t)AS_WARPS * cap) +
                    (size_t)warp * cap;
  for (int i = tid; i < 2 * d * d; i += AS_BLOCK) sU[i] = (Real)gp.U[i];
  for (int i = tid; i < 256; i += AS_BLOCK) (&s_inv[0][0])[i] = (&gp.perm->inv[0][0])[i];
  if (tid < 16) {
    s_re_nz[tid] = gp.re_nz[tid];
    s_im_nz[tid] = gp.im_nz[tid];
  }
  __syncthreads();
  const uint64_t G = ctl->count[0];
  const uint64_t imask = vb ? ((1ull << vb) - 1ull) : 0ull;
  uint32_t zeros = 0;
  for (uint64_t wb = (uint64_t)blockIdx.x * AS_WARPS + warp; wb * 32 < G; wb += (uint64_t)gridDim.x * AS_WARPS) {
    const uint64_t g = wb * 32 + lane;
    const bool valid = g < G;
    uint32_t h = 0, gmv = 0;
    uint64_t ob = 0;
    if (valid) {
      h = heads[g];
      gmv = gmask[g];
      ob = ooff[g];
    }
    const uint32_t pm = gmv & 0xffffu, om = gmv >> 16;
    const uint32_t s = (uint32_t)__popc(pm), c = (uint32_t)__popc(om);
    // members of the 32 groups, packed in group order
    uint32_t mx = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, mx, o);
      if (lane >= o) mx += y;
    }
    const uint32_t mb = mx - s;
    uint64_t rest = 0;
    for (uint32_t k = 0; k < s; ++k) {
      const uint64_t v = sk[h + k];
      if (k == 0) rest = v >> (m + vb);
      const uint64_t idx = vb ? (v & imask) : (uint64_t)sidx[h + k];
      xs[mb + k] = amps_in[idx];
    }
    // output slots ordered by member count, then by group
    uint32_t start = 0, T = 0;
    for (int l = 0; l < 32; ++l) {
      const uint32_t s2 = __shfl_sync(0xffffffffu, s, l), c2 = __shfl_sync(0xffffffffu, c, l);
      T += c2;
      if (s2 < s || (s2 == s && l < lane)) start += c2;
    }
    {
      uint32_t rem = om, k = 0;
      while (rem) {
        const uint32_t ro = (uint32_t)(__ffs(rem) - 1);
        rem &= rem - 1u;
        slots[start + k++] = (uint16_t)((lane << 4) | ro);
      }
    }
    __syncwarp();
    for (uint32_t b0 = 0; b0 < T; b0 += 32) {
      const uint32_t si = b0 + lane;
      const bool act = si < T;
      const uint32_t e = act ? slots[si] : 0u;
      const int gl = (int)(e >> 4);
      const uint32_t ro = e & 15u;
      const uint32_t pm_g = __shfl_sync(0xffffffffu, pm, gl);
      const uint32_t om_g = __shfl_sync(0xffffffffu, om, gl);
      const uint32_t mb_g = __shfl_sync(0xffffffffu, mb, gl);
      const uint64_t ob_g = __shfl_sync(0xffffffffu, ob, gl);
      const uint64_t rest_g = __shfl_sync(0xffffffffu, rest, gl);
      bool z = false;
      if (act) {
        const uint32_t rnz = s_re_nz[ro] & pm_g, inz = s_im_nz[ro] & pm_g;
        uint32_t cols = rnz | inz;
        Real re = (Real)0, im = (Real)0;
        while (cols) {
          const int r = __ffs(cols) - 1;
          cols &= cols - 1u;
          const C2 x = xs[mb_g + __popc(pm_g & ((1u << r) - 1u))];
          const Real ur = sU[2 * (ro * d + r)], ui = sU[2 * (ro * d + r) + 1];
          if ((rnz >> r) & 1u) {
            re = sfma(ur, x.x, re);
            im = sfma(ur, x.y, im);
          }
          if ((inz >> r) & 1u) {
            re = sfma(-ui, x.y, re);
            im = sfma(ui, x.x, im);
          }
        }
        const uint64_t o = ob_g + (uint64_t)__popc(om_g & ((1u << ro) - 1u));
        C2 y;
        y.x = re;
        y.y = im;
        keys_out[o] = permute_bits(s_inv, (rest_g << m) | ro);
        amps_out[o] = y;
        probs_out[o] = amp_prob_bits(y);
        z = is_zero_amp(re, im);
      }
      zeros += (uint32_t)__popc(__ballot_sync(0xffffffffu, z));
    }
    __syncwarp();
  }
  if (lane == 0 && zeros) atomicAdd((unsigned long long*)&ctl->count[3], (unsigned long long)zeros);
}

void launch_gate_apply_slots(int prec, const uint64_t* sk, const uint32_t* sidx, uint64_t n, const uint32_t* heads,
                             const uint32_t* gmask, const uint64_t* ooff, const void* amps_in, const GateParams& gp,
                             uint64_t* keys_out, void* amps_out, uint64_t* probs_out, Ctl* ctl, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_gate_apply_slots<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)slots_smem<double>(4));
    cudaFuncSetAttribute(k_gate_apply_slots<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)slots_smem<float>(4));
    attr_set = true;
  }
  cudaMemsetAsync(&ctl->count[3], 0, sizeof(uint64_t), st);
  if (n == 0) return;
  const uint64_t batches = (n + 31) / 32;  // groups <= n
  uint64_t grid = (batches + AS_WARPS - 1) / AS_WARPS;
  if (grid > 148ull * 4) grid = 148ull * 4;
  if (prec == 0)
    k_gate_apply_slots<double><<<(unsigned)grid, AS_BLOCK, slots_smem<double>(gp.m), st>>>(
        sk, sidx, heads, gmask, ooff, (const double2*)amps_in, gp, keys_out, (double2*)amps_out, probs_out, ctl);
  else
    k_gate_apply_slots<float><<<(unsigned)grid, AS_BLOCK, slots_smem<float>(gp.m), st>>>(
        sk, sidx, heads, gmask, ooff, (const float2*)amps_in, gp, keys_out, (float2*)amps_out, probs_out, ctl);
}

}  // namespace sv
