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
//   * k_gate_apply_slots: a warp takes a batch of groups, stages their
//     members' amplitudes in shared memory, orders the groups' output slots
//     by member count (so the lanes of a round run chains of equal length), and each
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
#include "launch.cuh"
#include "select.cuh"
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
  pdl_prologue();
  extern __shared__ __align__(16) uint8_t s_dyn[];
  uint64_t* s_k = reinterpret_cast<uint64_t*>(s_dyn);
  __shared__ uint32_t s_wh[GS_WARPS], s_wo[GS_WARPS], s_colnz[16];
  __shared__ bool s_dense;
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
  if (tid == 0) {  // every column of U nonzero in every row
    bool dense = true;
    for (int r = 0; r < (1 << m); ++r)
      for (int ro = 0; ro < (1 << m); ++ro)
        if (!(((gp.re_nz[ro] | gp.im_nz[ro]) >> r) & 1u)) dense = false;
    s_dense = dense;
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
    // stage the tile and its halo, eight loads per thread in flight at a time
#pragma unroll
    for (int h = 0; h < GS_ITEMS; h += 8) {
      uint64_t r[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int e = tid + (h + j) * GS_BLOCK;
        r[j] = e < staged ? sk[base + e] : 0ull;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int e = tid + (h + j) * GS_BLOCK;
        if (e < staged) s_k[e + 1] = r[j];
      }
    }
    if (tid < GS_HALO && GS_TILE + tid < staged) s_k[GS_TILE + tid + 1] = sk[base + GS_TILE + tid];
    __syncthreads();
    const int wbase = warp * 32 * GS_ITEMS;
    // pass 1: the warp's head and output counts (for a U without zero
    // entries every group has all 2^m outputs: the heads alone decide)
    uint32_t nh = 0, no = 0;
    if (s_dense) {
#pragma unroll 4
      for (int j = 0; j < GS_ITEMS; ++j) {
        const int e = wbase + j * 32 + lane;
        const bool f = e < tn && (s_k[e] >> shift) != (s_k[e + 1] >> shift);
        nh += (uint32_t)__popc(__ballot_sync(0xffffffffu, f));
      }
      no = nh << m;
    } else {
#pragma unroll 4
      for (int j = 0; j < GS_ITEMS; ++j) {
        const int e = wbase + j * 32 + lane;
        uint32_t pm, om;
        const bool f = e < tn && gs_head(s_k, e, staged, shift, vb, dmask, s_colnz, pm, om);
        nh += (uint32_t)__popc(__ballot_sync(0xffffffffu, f));
        no += __reduce_add_sync(0xffffffffu, f ? (uint32_t)__popc(om) : 0u);
      }
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
        if (!s_dense) ooff[gi] = o + (cx - c);  // dense U: group g starts at g 2^m
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

uint64_t group_scan_lookback_words(uint64_t n) { return 2 * (n / GS_TILE + 2); }

void launch_group_scan(const uint64_t* sk, uint64_t n, const GateParams& gp, uint32_t* heads, uint32_t* gmask,
                       uint64_t* ooff, uint64_t* lookback, Ctl* ctl, cudaStream_t st) {
  (void)slots_prepare();  // checked at the handle's creation; a launch without it fails loudly
  const uint64_t tiles = (n + GS_TILE - 1) / GS_TILE;
  // the look-back words, ctl->tile_counter[0] and ctl->count[0..1] arrive
  // cleared (the gate's table upload clears them)
  if (n == 0) return;
  const uint64_t grid = tiles < 148 * 3 ? tiles : 148 * 3;
  launch_pdl(k_group_scan, (unsigned)grid, GS_BLOCK, GS_SMEM, st, sk, n, gp, heads, gmask, ooff, lookback,
             lookback + tiles + 1, ctl);
}

// A warp takes a batch of 32 * gpl groups.  Larger batches leave fewer
// rounds whose lanes run chains of different lengths; smaller ones leave
// room for more warps per SM and, with batches taken from a counter, balance
// better (measured at m = 2: gpl = 2 for both precisions, against 4 and 1
// for complex64 and 1 for complex128, which is bound by the FP64 pipe; the
// batch halves again above m = 2).  A batch holds at most 32 * gpl * 2^m
// members and output slots.
constexpr int AS_WARPS = 8, AS_BLOCK = AS_WARPS * 32;
constexpr int AS_UNROLL = 4;  // member loads in flight per lane

__host__ __device__ __forceinline__ int slots_gpl(int prec, int m) {
  return prec == 0 ? (m <= 3 ? 2 : 1) : (m <= 2 ? 2 : 1);
}

// Per-warp shared layout of a batch of GC = 32 * gpl groups and MC = GC * 2^m
// members: x[MC] (amplitudes), ob[GC], rest[GC], pmom[GC], mb[GC], sst[GC],
// slots[MC], oc[GC].
template <typename C2>
struct SlotsLayout {
  C2* x;
  uint64_t *ob, *rest;
  uint32_t* pmom;
  uint16_t *mb, *sst, *slots;
  uint8_t* oc;
  __host__ __device__ static size_t bytes(uint32_t gc, uint32_t mc) {
    const size_t b = (size_t)mc * sizeof(C2) + (size_t)gc * (8 + 8 + 4 + 2 + 2 + 1) + (size_t)mc * 2;
    return (b + 15) & ~(size_t)15;
  }
  __device__ SlotsLayout(uint8_t* base, uint32_t gc, uint32_t mc) {
    x = reinterpret_cast<C2*>(base);
    ob = reinterpret_cast<uint64_t*>(base + (size_t)mc * sizeof(C2));
    rest = ob + gc;
    pmom = reinterpret_cast<uint32_t*>(rest + gc);
    mb = reinterpret_cast<uint16_t*>(pmom + gc);
    sst = mb + gc;
    slots = sst + gc;
    oc = reinterpret_cast<uint8_t*>(slots + mc);
  }
};

// complex128 at four blocks per SM (64 registers); complex64 without a
// minimum (0: the compiler's own register choice, 40-48, which measured
// fastest for the float kernel)
template <typename Real, int GPL>
__global__ void __launch_bounds__(AS_BLOCK, sizeof(Real) == 8 ? 4 : 0) k_gate_apply_slots(
    const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sidx, const uint32_t* __restrict__ heads,
    const uint32_t* __restrict__ gmask, const uint64_t* __restrict__ ooff,
    const typename SCplx<Real>::T* __restrict__ amps_in, const GateParams gp, uint64_t* __restrict__ keys_out,
    typename SCplx<Real>::T* __restrict__ amps_out, uint64_t* __restrict__ probs_out, Ctl* ctl) {
  pdl_prologue();
  constexpr int gpl = GPL;
  typedef typename SCplx<Real>::T C2;
  extern __shared__ __align__(16) uint8_t s_dyn[];
  // U with its rows padded to d + 1 entries: the lanes of a round read
  // U[r'][r] for different r' and mostly the same r, which the padding puts
  // in different banks
  __shared__ Real sU[2 * 16 * 17];
  __shared__ uint32_t s_re_nz[16], s_im_nz[16];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const int m = gp.m, d = 1 << m, vb = gp.vbits, shift = m + vb;
  const uint32_t gc = 32u * gpl, mc = gc << m;
  SlotsLayout<C2> w(s_dyn + (size_t)warp * SlotsLayout<C2>::bytes(gc, mc), gc, mc);
  for (int i = tid; i < 2 * d * d; i += AS_BLOCK) {
    const int e = i >> 1, ro = e >> m, r = e & (d - 1);
    sU[2 * (ro * (d + 1) + r) + (i & 1)] = (Real)gp.U[i];
  }
  if (tid < 16) {
    s_re_nz[tid] = gp.re_nz[tid];
    s_im_nz[tid] = gp.im_nz[tid];
  }
  // no zero entry in U: every group has all 2^m outputs, group g's first at
  // g 2^m (the group scan then writes no output positions)
  const uint32_t full = (1u << d) - 1u;
  const bool dense = __syncthreads_and(tid >= d || ((gp.re_nz[tid & 15] | gp.im_nz[tid & 15]) & full) == full);
  const uint64_t G = ctl->count[0];
  const uint64_t imask = vb ? ((1ull << vb) - 1ull) : 0ull;
  uint32_t zeros = 0;
  // complex128: the exact fixed-point total mass of the candidates, summed on
  // the integer pipe while the FP64 pipe does the multiply-adds (the
  // truncation's window pass then needs no per-term mass for a top-K cut)
  constexpr bool MASS = sizeof(Real) == 8;
  constexpr bool COALESCED = sizeof(Real) == 8;
  u128 tot = 0;
  // batches are taken from a counter (ctl->tile_counter[1], cleared with the
  // gate's tables): warps whose groups have more members take fewer batches
  uint64_t wb = 0;
  if (lane == 0) wb = atomicAdd((unsigned long long*)&ctl->tile_counter[1], 1ull);
  wb = __shfl_sync(0xffffffffu, wb, 0);
  for (; wb * gc < G;) {
    // group j = 32 k + lane of the batch; all group loads first
    uint32_t s[GPL], c[GPL], pos[GPL], h[GPL], gmv[GPL];
    uint64_t ob[GPL];
#pragma unroll
    for (int k = 0; k < GPL; ++k) {
      h[k] = 0;
      gmv[k] = 0;
      ob[k] = 0;
      const uint64_t g = wb * gc + 32 * k + lane;
      if (k < gpl && g < G) {
        h[k] = heads[g];
        gmv[k] = gmask[g];
        ob[k] = dense ? g << m : ooff[g];
      }
    }
    uint32_t mrun = 0, ng = 0, mb[GPL];
#pragma unroll
    for (int k = 0; k < GPL; ++k) {
      s[k] = (uint32_t)__popc(gmv[k] & 0xffffu);
      c[k] = (uint32_t)__popc(gmv[k] >> 16);
      uint32_t mx = s[k];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, mx, o);
        if (lane >= o) mx += y;
      }
      mb[k] = mrun + mx - s[k];
      mrun += __shfl_sync(0xffffffffu, mx, 31);
      ng += (uint32_t)__popc(__ballot_sync(0xffffffffu, s[k] != 0));
    }
    // Each group's first key gives its rest.  complex128: the batch's groups
    // are consecutive in the grouped order, so their members are the mrun
    // terms from the first group's head on, member t of group j at mb[j] + t:
    // all lanes load them together (coalesced keys or indices, then the
    // amplitude gathers, AS_UNROLL of each in flight).  complex64 (measured
    // faster at its higher occupancy): each lane loads its groups' members.
    uint64_t rest[GPL];
#pragma unroll
    for (int k = 0; k < GPL; ++k) rest[k] = s[k] ? sk[h[k]] : 0ull;
    if (COALESCED) {
      const uint64_t e0 = __shfl_sync(0xffffffffu, (uint64_t)h[0], 0);  // head of group wb * gc (< G)
      for (uint32_t i0 = 0; i0 < mrun; i0 += 32u * AS_UNROLL) {
        uint64_t src[AS_UNROLL];
#pragma unroll
        for (int u = 0; u < AS_UNROLL; ++u) {
          const uint32_t i = i0 + 32u * u + lane;
          src[u] = 0;
          if (i < mrun) src[u] = vb ? (sk[e0 + i] & imask) : (uint64_t)sidx[e0 + i];
        }
        C2 xv[AS_UNROLL];
#pragma unroll
        for (int u = 0; u < AS_UNROLL; ++u)
          if (i0 + 32u * u + lane < mrun) xv[u] = amps_in[src[u]];
#pragma unroll
        for (int u = 0; u < AS_UNROLL; ++u)
          if (i0 + 32u * u + lane < mrun) w.x[i0 + 32u * u + lane] = xv[u];
      }
    }
#pragma unroll
    for (int k = 0; k < GPL; ++k) {
      if (!s[k]) continue;
      const uint64_t v0 = rest[k];
      if (!COALESCED) {
        w.x[mb[k]] = amps_in[vb ? (v0 & imask) : (uint64_t)sidx[h[k]]];
        for (uint32_t t = 1; t < s[k]; ++t) {
          const uint64_t v = sk[h[k] + t];
          w.x[mb[k] + t] = amps_in[vb ? (v & imask) : (uint64_t)sidx[h[k] + t]];
        }
      }
      const uint32_t j = 32u * k + lane;
      w.pmom[j] = gmv[k];
      w.mb[j] = (uint16_t)mb[k];
      w.ob[j] = ob[k];
      w.rest[j] = v0 >> shift;
    }
    // order the groups by member count (ballots per count), then give each
    // ordered position its first slot (scan of the output counts)
    uint32_t cnt = 0;
    for (int v = 1; v <= d; ++v) {
#pragma unroll
      for (int k = 0; k < GPL; ++k) {
        if (k >= gpl) continue;
        const bool hit = s[k] == (uint32_t)v;
        const uint32_t b = __ballot_sync(0xffffffffu, hit);
        if (hit) pos[k] = cnt + (uint32_t)__popc(b & lt);
        cnt += (uint32_t)__popc(b);
      }
    }
#pragma unroll
    for (int k = 0; k < GPL; ++k)
      if (k < gpl && s[k]) w.oc[pos[k]] = (uint8_t)c[k];
    __syncwarp();
    {
      uint32_t loc[GPL], sum = 0;
#pragma unroll
      for (int i = 0; i < GPL; ++i) {
        const uint32_t p = (uint32_t)lane * gpl + i;
        loc[i] = (i < gpl && p < ng) ? w.oc[p] : 0u;
        sum += loc[i];
      }
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      uint32_t run = x - sum;
#pragma unroll
      for (int i = 0; i < GPL; ++i) {
        const uint32_t p = (uint32_t)lane * gpl + i;
        if (i < gpl && p < ng) w.sst[p] = (uint16_t)run;
        run += loc[i];
      }
    }
    __syncwarp();
    uint32_t T = 0;
#pragma unroll
    for (int k = 0; k < GPL; ++k) {
      if (k >= gpl) continue;
      T += __reduce_add_sync(0xffffffffu, c[k]);
      if (s[k]) {
        const uint32_t j = 32u * k + lane;
        uint32_t rem = w.pmom[j] >> 16, st = w.sst[pos[k]];
        while (rem) {
          const uint32_t ro = (uint32_t)(__ffs(rem) - 1);
          rem &= rem - 1u;
          w.slots[st++] = (uint16_t)((j << 4) | ro);
        }
      }
    }
    __syncwarp();
    for (uint32_t b0 = 0; b0 < T; b0 += 32) {
      const uint32_t si = b0 + lane;
      bool z = false;
      if (si < T) {
        const uint32_t e = w.slots[si];
        const uint32_t j = e >> 4, ro = e & 15u;
        const uint32_t pmom = w.pmom[j], pm_g = pmom & 0xffffu, om_g = pmom >> 16;
        const uint32_t mb_g = w.mb[j];
        const uint32_t rnz = s_re_nz[ro] & pm_g, inz = s_im_nz[ro] & pm_g;
        uint32_t cols = rnz | inz;
        Real re = (Real)0, im = (Real)0;
        while (cols) {
          const int r = __ffs(cols) - 1;
          cols &= cols - 1u;
          const C2 x = w.x[mb_g + __popc(pm_g & ((1u << r) - 1u))];
          const Real ur = sU[2 * (ro * (d + 1) + r)], ui = sU[2 * (ro * (d + 1) + r) + 1];
          if ((rnz >> r) & 1u) {
            re = sfma(ur, x.x, re);
            im = sfma(ur, x.y, im);
          }
          if ((inz >> r) & 1u) {
            re = sfma(-ui, x.y, re);
            im = sfma(ui, x.x, im);
          }
        }
        const uint64_t o = w.ob[j] + (uint64_t)__popc(om_g & ((1u << ro) - 1u));
        C2 y;
        y.x = re;
        y.y = im;
        keys_out[o] = (w.rest[j] << m) | ro;  // outputs are stored in the gate's sort-key order
        amps_out[o] = y;
        const uint64_t pb = amp_prob_bits(y);
        probs_out[o] = pb;
        if (MASS) tot += fx_from_bits(pb, &ctl->err);
        z = is_zero_amp(re, im);
      }
      zeros += (uint32_t)__popc(__ballot_sync(0xffffffffu, z));
    }
    __syncwarp();
    if (lane == 0) wb = atomicAdd((unsigned long long*)&ctl->tile_counter[1], 1ull);
    wb = __shfl_sync(0xffffffffu, wb, 0);
  }
  if (lane == 0 && zeros) atomicAdd((unsigned long long*)&ctl->count[3], (unsigned long long)zeros);
  if (MASS) {
    tot = warp_sum_u128(tot);
    if (lane == 0 && tot) atomic_add_u128(&ctl->total_mass_hi, &ctl->total_mass_lo, tot);
  }
}

// Resident blocks per SM of the slot mat-vec, by device, precision and m
// (set by slots_prepare).
int g_slots_occ[DeviceOnce::kMaxDevices][2][5];

template <typename R, int GPLV, typename C2>
cudaError_t slots_setup(int dev, int prec) {
  // the largest batch of any m that uses this variant: 32 * GPLV groups, 512 members
  cudaError_t e = cudaFuncSetAttribute(k_gate_apply_slots<R, GPLV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(AS_WARPS * SlotsLayout<C2>::bytes(32 * GPLV, 512)));
  for (int m = 1; m <= 4 && e == cudaSuccess; ++m) {
    if (slots_gpl(prec, m) != GPLV) continue;
    const uint32_t gc = 32u * GPLV, mc = gc << m;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gate_apply_slots<R, GPLV>, AS_BLOCK,
                                                      AS_WARPS * SlotsLayout<C2>::bytes(gc, mc));
    g_slots_occ[dev][prec][m] = per_sm;
  }
  return e;
}

cudaError_t slots_prepare() {
  static DeviceOnce once;
  return once.run([] {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_group_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GS_SMEM);
    if (e == cudaSuccess) e = slots_setup<double, 2, double2>(dev, 0);
    if (e == cudaSuccess) e = slots_setup<double, 1, double2>(dev, 0);
    if (e == cudaSuccess) e = slots_setup<float, 4, float2>(dev, 1);
    if (e == cudaSuccess) e = slots_setup<float, 2, float2>(dev, 1);
    if (e == cudaSuccess) e = slots_setup<float, 1, float2>(dev, 1);
    return e;
  });
}

void launch_gate_apply_slots(int prec, const uint64_t* sk, const uint32_t* sidx, uint64_t n, const uint32_t* heads,
                             const uint32_t* gmask, const uint64_t* ooff, const void* amps_in, const GateParams& gp,
                             uint64_t* keys_out, void* amps_out, uint64_t* probs_out, Ctl* ctl, cudaStream_t st) {
  const int gpl = slots_gpl(prec, gp.m);
  const uint32_t gc = 32u * gpl, mc = gc << gp.m;
  const size_t smem = AS_WARPS * (prec == 0 ? SlotsLayout<double2>::bytes(gc, mc) : SlotsLayout<float2>::bytes(gc, mc));
  // ctl->count[3] and the total mass arrive cleared (the gate's table upload)
  if (n == 0) return;
  const uint64_t batches = (n + gc - 1) / gc;  // groups <= n
  uint64_t grid = (batches + AS_WARPS - 1) / AS_WARPS;
  (void)slots_prepare();  // checked at the handle's creation; a launch without it fails loudly
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= DeviceOnce::kMaxDevices) dev = 0;
  int per_sm = g_slots_occ[dev][prec ? 1 : 0][gp.m];
  if (per_sm < 1) per_sm = 1;
#define SV_SLOTS(R, C2, GPLV)                                                                                 \
  do {                                                                                                        \
    if (grid > 148ull * per_sm) grid = 148ull * per_sm;                                                       \
    /* ordinary launch: scheduled early behind the group scan it ran slower with static batches, no faster now */ \
    k_gate_apply_slots<R, GPLV><<<(unsigned)grid, AS_BLOCK, smem, st>>>(sk, sidx, heads, gmask, ooff,           \
                                                                        (const C2*)amps_in, gp, keys_out,        \
                                                                        (C2*)amps_out, probs_out, ctl);          \
  } while (0)
  if (prec == 0) {
    if (gpl == 2)
      SV_SLOTS(double, double2, 2);
    else
      SV_SLOTS(double, double2, 1);
  } else {
    if (gpl == 4)
      SV_SLOTS(float, float2, 4);
    else if (gpl == 2)
      SV_SLOTS(float, float2, 2);
    else
      SV_SLOTS(float, float2, 1);
  }
#undef SV_SLOTS
}

}  // namespace sv
