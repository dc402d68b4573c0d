// Internal launch interfaces between the translation units of libsv.so.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace sv {

constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int MAX_PASSES = 8;
constexpr int SORT_THREADS = 512;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;

// Scratch used by one LSD radix sort.
struct SortScratch {
  uint32_t* hist;        // [MAX_PASSES][RADIX] device digit counts
  uint32_t* hist_host;   // pinned mirror of hist
  uint64_t* lookback;    // [tiles][RADIX] look-back descriptors for one pass
  uint64_t lookback_tiles;
  uint64_t* tile_counter;
  uint32_t* err;
};

inline uint64_t sort_tiles(uint64_t n) { return (n + SORT_TILE - 1) / SORT_TILE; }

// Histogram of every 8-bit digit of k[0..n) over the low nbits bits.
void launch_digit_hist(const uint64_t* k, uint64_t n, int nbits, uint32_t* hist, cudaStream_t st);

// Stable LSD radix sort of (k, v) pairs on bits [0, nbits) of k, with the
// digit histograms already in scratch.hist (and its host mirror when
// hist_on_host).  Passes whose digit is constant over all keys are skipped.
// The result lands in (kA, vA) when the return value is 0, in (kB, vB)
// when it is 1.  *passes_run receives the number of scatter passes.
// Keys-only LSD sort on the bits [lo, lo + nbits) of each key (bits below lo
// ride along, e.g. a packed index); histograms in sc.hist are of the digits
// of key >> lo.  Returns the buffer holding the result (0: kA, 1: kB).
int radix_sort_keys(uint64_t* kA, uint64_t* kB, uint64_t n, int lo, int nbits, const SortScratch& sc,
                    cudaStream_t st, int* passes_run, cudaError_t* cerr);
cudaError_t sort_prepare();
int radix_sort_pairs(uint64_t* kA, uint32_t* vA, uint64_t* kB, uint32_t* vB, uint64_t n, int nbits,
                     const SortScratch& sc, cudaStream_t st, int* passes_run, cudaError_t* cerr);

// Exclusive scan over tiles of per-tile digit counts cnt[d * tiles + t]
// for digits d < digits, each digit's run starting after the smaller
// digits' totals (hist[d]): off[d * tiles + t].
void launch_tile_offsets(const uint32_t* cnt, const uint32_t* hist, uint64_t tiles, int digits, uint32_t* off,
                         cudaStream_t st);

// Stored keys.  The state keeps its terms sorted by the sort key of the last
// gate, and it stores each term's key in that sort key's bit order (the
// qubit order): bit order[b] of a stored key is qubit b.  Natural keys
// (qubit i = bit i) are produced only where they leave the library or decide
// canonical order: readouts, and probability ties at a cut or a peak.
//
// Sort-key bit permutation of a gate, on stored keys: the gate qubits go to
// the bottom with qubits[t] at bit t, the other bits keep their order above
// them.  Equal (sort key >> m) <=> same partner group, with members in
// ascending r.  The gate's outputs are stored in the new order, so inv (new
// sort key -> new stored key) is the identity.
struct BitPerm {
  uint64_t fwd[16][16];  // stored key -> sort key
  uint64_t inv[16][16];  // sort key -> stored key of the outputs
};

// Per-gate tables uploaded once per gate (one copy) and read by the kernels
// through the pointers in GateParams, which stays small enough to pass by
// value cheaply.  nat maps the stored keys of the gate's outputs to natural
// keys; it stays valid until the next gate.
struct GateTables {
  BitPerm perm;
  uint64_t nat[16][16];
  double U[512];
};

// Per-gate counters cleared by the table upload of a gate on the global path
// (one launch instead of a memset per counter): ctl->tile_counter[0..1],
// ctl->count[0..3], the total mass, the 16 partition totals of the
// regrouping and the group scan's look-back words.  ctl == nullptr: none.
struct GateReset {
  Ctl* ctl;
  uint32_t* part_hist;  // [16]
  uint64_t* lb;         // [lb_words]
  uint32_t lb_words;
};

// Stores the first `bytes` bytes of t (passed by value) at dst and clears
// what r names.
void launch_store_tables(const GateTables& t, GateTables* dst, size_t bytes, const GateReset& r, cudaStream_t st);

// Gate parameters passed by value to the gate kernels.
struct GateParams {
  uint64_t qmask;
  uint64_t n_mask;
  int m;
  int q[4];            // gate qubits in the caller's order (bit t of r)
  int qs[4];           // the same qubits in ascending order
  uint32_t re_nz[16];  // bit r set when Re U[r_out][r] != 0
  uint32_t im_nz[16];  // bit r set when Im U[r_out][r] != 0
  const double* U;     // device copy of U[r_out][r] as (re, im), row-major
  const BitPerm* perm; // device copy of this gate's sort-key permutation
  int n;               // qubits
  int tbits;           // number of bucket qubits (top bits of the sort key)
  uint64_t pmask;      // bucket qubits as a key mask
  int vbits;           // > 0: sort keys carry the term index in their low vbits bits (no index array)
  int qpos[4];         // bit of qubits[t] in the stored keys before the gate
  uint64_t rmap;       // nibble r: the digit the regrouping sorts a term with gate bits r under
                       // (identity; a monomial gate's output index instead)
  int direct;          // 1: the keys given to the regrouping are already sort keys (digit = low m
                       // bits; a key of all ones is left out), as in the batched form
};

constexpr uint64_t RMAP_IDENTITY = 0xFEDCBA9876543210ull;

// Natural key of a stored key, with the nibble table of GateTables::nat
// (256 entries, in shared or global memory).
__device__ __forceinline__ uint64_t to_natural(const uint64_t* nat, uint64_t x) {
  uint64_t y = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) y |= nat[16 * k + ((x >> (4 * k)) & 15u)];
  return y;
}

// Grouping of a state that is sorted by the previous gate's sort key when
// gp.perm keeps the other qubits in that order (gate qubits at the bottom):
// stable partition by the gate bits r, then m levels of pairwise merges.
// The sorted keys (packed with the term index when gp.vbits > 0, else with
// indices in sidx) end in sk[w], w the return value; *launches receives
// the number of kernels launched.  The scratch's lookback words hold the
// per-tile counts and offsets, hist the counts per r (its first 16 words
// cleared beforehand: GateReset::part_hist).
int regroup_terms(const uint64_t* keys, uint64_t n, const GateParams& gp, uint64_t* sk[2], uint32_t* sidx[2],
                  const SortScratch& sc, cudaStream_t st, int* launches, cudaError_t* cerr);
cudaError_t regroup_prepare();
// Kernel attributes (dynamic shared-memory limits) and launch-shape tables
// of this device, set once per device; the handles' creation checks them.
cudaError_t slots_prepare();
cudaError_t local_prepare();
cudaError_t select_prepare();

// Expand-first gate application (Sec. IV-A as the paper states it): records
// (output sort key << m | source r, source index) for every term and output,
// and the per-output reduction over the sorted records.
void launch_expand_records(const uint64_t* keys, uint64_t n, const GateParams& gp, uint64_t* sk, uint32_t* sidx,
                           uint32_t* hist, int passes, cudaStream_t st);
void launch_segment_reduce(int prec, const uint64_t* sk, const uint32_t* sidx, uint64_t nrec, const uint32_t* heads,
                           const void* amps_in, const GateParams& gp, uint64_t* keys_out, void* amps_out,
                           uint64_t* probs_out, uint64_t* lookback, Ctl* ctl, uint64_t max_tiles, cudaStream_t st);

void launch_gate_keys(const uint64_t* keys, uint64_t n, const GateParams& gp, uint64_t* sk,
                      uint32_t* sv_out, uint32_t* hist, int passes, cudaStream_t st);

// Mark partner-group heads of the grouped sequence and compact their
// positions; the group count lands in ctl->count[0].
void launch_group_heads(const uint64_t* sk, uint64_t n, int shift, uint32_t* heads, uint64_t* lookback,
                        Ctl* ctl, cudaStream_t st);

// Partner-group heads of the grouped sort keys with, per group, the present
// mask pm (bit r: member with gate bits r present) | output mask om << 16
// (bit r': some present r meets a nonzero U[r'][r]) in gmask, and the
// group's first output position (exclusive scan of popc(om)) in ooff, which
// is left unwritten when U has no zero entry (group g then starts at g 2^m).
// Group count in ctl->count[0], candidate count in ctl->count[1].  Uses
// group_scan_lookback_words(n) lookback words, which, with
// ctl->tile_counter[0] and ctl->count[0..1], must be zero on entry
// (GateReset).
void launch_group_scan(const uint64_t* sk, uint64_t n, const GateParams& gp, uint32_t* heads, uint32_t* gmask,
                       uint64_t* ooff, uint64_t* lookback, Ctl* ctl, cudaStream_t st);
// Look-back words launch_group_scan uses for n terms (both look-backs).
uint64_t group_scan_lookback_words(uint64_t n);
// Per-group mat-vec writing each structurally nonzero output at its
// precomputed position; exact zeros are written as zero and counted in
// ctl->count[3] (to be removed by launch_drop_zero_terms).  complex128 also
// sums the candidates' exact fixed-point total mass into ctl->total_mass.
// ctl->count[3], the total mass and ctl->tile_counter[1] (the batch counter)
// must be zero on entry (GateReset).
void launch_gate_apply_slots(int prec, const uint64_t* sk, const uint32_t* sidx, uint64_t n, const uint32_t* heads,
                             const uint32_t* gmask, const uint64_t* ooff, const void* amps_in, const GateParams& gp,
                             uint64_t* keys_out, void* amps_out, uint64_t* probs_out, Ctl* ctl, cudaStream_t st);

// Local gate on a bucket-contiguous state (no bucket qubit in the gate):
// each block takes the buckets that start in its chunk, sorts them in
// shared memory by the gate's sort key, and writes its outputs into one
// atomically reserved range sized by the structurally nonzero outputs.
// The library uses it with no bucket qubits for states of at most
// LOCAL_BUCKET_MAX terms (one block does the whole gate).
// Exact-zero outputs that the structure did not predict are written with a
// zero amplitude and counted in ctl->count[3] (removed by
// launch_drop_zero_terms).  Output count in ctl->count[1]; a bucket larger
// than the batch limit sets ERR_BUCKET.
constexpr int LOCAL_CHUNK = 4096;
constexpr int LOCAL_CAP = 8192;
constexpr uint64_t LOCAL_BUCKET_MAX = LOCAL_CAP - LOCAL_CHUNK;
void launch_local_gate(int prec, const uint64_t* keys, const void* amps, uint64_t n, const GateParams& gp,
                       uint64_t* keys_out, void* amps_out, uint64_t* probs_out, Ctl* ctl, cudaStream_t st);
// Order-preserving removal of zero-amplitude terms (count in ctl->count[2]).
// A diagonal gate applied in place (csrc/diag.cu): ur/ui[r] = U[r][r],
// rnz/inz bit r set when its real / imaginary part is nonzero (complex64:
// after rounding to float), qpos[t] the stored bit of qubits[t].  The term
// order and keys are unchanged; amps and probs are overwritten, the exact
// total mass is added into ctl->total_mass and exact zeros are counted in
// ctl->count[3] (both must be zero on entry).
struct DiagParams {
  double ur[16], ui[16];
  uint32_t rnz, inz;
  uint32_t unit, uneg;  // bit r: entry r is +-1 or +-i; its nonzero component is -1
  int m;
  int qpos[4];
};
void launch_diag_apply(int prec, const uint64_t* keys, void* amps, uint64_t* probs, uint64_t n, const DiagParams& dp,
                       Ctl* ctl, cudaStream_t st);

// A monomial gate (one nonzero per row and column: permutations with
// phases, e.g. X, CNOT, Toffoli, C3X): the regrouping sorted the terms by
// their output key (GateParams::rmap = the gate's output index of each r),
// so output i is sk[i]'s term times its one matrix entry.  ur/ui[r'] =
// U[r'][r] for the r mapped to r', rnz/inz bit r' set when nonzero (after
// rounding to float for complex64).  Writes N outputs in order, the exact
// total mass into ctl->total_mass and the exact zeros into ctl->count[3]
// (both zero on entry).
struct MonoParams {
  double ur[16], ui[16];
  uint32_t rnz, inz;
  uint32_t unit, uneg;  // as in DiagParams, by output index r'
  int m, vbits;
};
void launch_mono_apply(int prec, const uint64_t* sk, const uint32_t* sidx, uint64_t n, const void* amps_in,
                       const MonoParams& mp, uint64_t* keys_out, void* amps_out, uint64_t* probs_out, Ctl* ctl,
                       cudaStream_t st);

void launch_drop_zero_terms(int prec, const uint64_t* keys, const void* amps, const uint64_t* probs,
                            uint64_t n, uint64_t* keys_out, void* amps_out, uint64_t* probs_out,
                            uint64_t* lookback, Ctl* ctl, cudaStream_t st);

// Truncation select.
constexpr int SEL_BITS = 11;
constexpr int SEL_BINS = 1 << SEL_BITS;
constexpr int FINISH_CAP = 4096;

struct SelectScratch {
  uint32_t* hist_count;   // [SEL_BINS]
  uint64_t* hist_mass;    // [SEL_BINS][2] (hi, lo)
  uint64_t* buf;          // [FINISH_CAP][2] composite (hi = ~pbits, lo = key)
  uint64_t* win_p;        // [win_cap] probability bits of the window terms
  uint32_t* win_i;        // [win_cap] positions of the window terms (their keys stay in place)
  uint64_t win_cap;
  uint32_t* tile_keep;    // [window tiles] kept terms per tile
  uint64_t* tile_off;     // [window tiles] output offset per tile
  uint32_t* keep_bits;    // [window tiles * WINDOW_TILE / 32] keep flag of every term
  uint64_t tiles_cap;
};
constexpr int WINDOW_TILE = 2048;  // terms per tile of the window pass and windowed compaction

// Number of tiles of the window pass (and of the windowed compaction).
uint64_t window_tiles(uint64_t n);
// After a select on the window: per-tile kept counts, their scan (total in
// ctl->count[2]) and the lookback-free renormalising compaction.
// The compactions leave each block's canonical best kept term in
// peak_part[2b], peak_part[2b + 1] (probability bits, key) for blocks
// b < *peak_blocks <= PEAK_PARTS; launch_peak_partials reduces them.  They
// write keys and rescaled amplitudes only: the kept terms' new
// probabilities are computed where a term can be its block's peak, and a
// caller that needs them all afterwards recomputes them (launch_amp_probs).
constexpr uint32_t PEAK_PARTS = 148 * 8;
void launch_truncate_windowed(int prec, const uint64_t* keys, const void* amps, const uint64_t* probs,
                              uint64_t n, uint64_t* keys_out, void* amps_out, const SelectScratch& ss, Ctl* ctl,
                              cudaStream_t st, uint64_t* peak_part, uint32_t* peak_blocks);
// probs[i] = the probability bits of amplitude i (its precision's formula).
void launch_amp_probs(int prec, const void* amps, uint64_t n, uint64_t* probs, cudaStream_t st);

// Sample-estimated window, one streaming pass (exact total mass, count and
// mass above the window, window terms gathered) and the choice of the list
// the radix select runs on (ctl->use_window); sets the select state.
// have_total: ctl->total_mass already holds the exact total of the terms
// (summed by the complex128 mat-vec); a top-K cut then skips it per term.
void launch_select_window(const uint64_t* probs, const uint64_t* keys, uint64_t n, Ctl* ctl,
                          const SelectScratch& ss, int mode, uint64_t count_target, double p,
                          bool have_total, cudaStream_t st);

void launch_select_hist(const uint64_t* probs, const uint64_t* keys, uint64_t n, Ctl* ctl,
                        const SelectScratch& ss, cudaStream_t st);
void launch_select_pick(Ctl* ctl, const SelectScratch& ss, double p, cudaStream_t st);
void launch_select_compact(const uint64_t* probs, const uint64_t* keys, uint64_t n, Ctl* ctl,
                           const SelectScratch& ss, cudaStream_t st);
void launch_select_finish(Ctl* ctl, const SelectScratch& ss, double p, cudaStream_t st);
// Keep the terms not after the cut in canonical order, scale them by
// ctl->scale and recompute their probabilities; count in ctl->count[2].
void launch_truncate_compact(int prec, const uint64_t* keys, const void* amps, const uint64_t* probs,
                             uint64_t n, uint64_t* keys_out, void* amps_out, uint64_t* lookback, Ctl* ctl,
                             cudaStream_t st, uint64_t* peak_part, uint32_t* peak_blocks);
void launch_peak_partials(const uint64_t* part, uint32_t n, Ctl* ctl, cudaStream_t st);
void launch_set_scale(Ctl* ctl, cudaStream_t st);
// Select state of one histogram level over all terms (prefix of `bits` fixed
// composite bits), and a cut at the composite (~pc, kc) with kept mass S_c.
void launch_set_select(Ctl* ctl, uint64_t ph, uint64_t pl, uint32_t bits, cudaStream_t st);
void launch_set_cut(Ctl* ctl, uint64_t pc, uint64_t kc, uint64_t sc_hi, uint64_t sc_lo, cudaStream_t st);

// Readout.
void launch_peak(const uint64_t* probs, const uint64_t* keys, uint64_t n, Ctl* ctl, cudaStream_t st);
void launch_iota(uint32_t* v, uint64_t n, cudaStream_t st);
void launch_not_bits_gather(const uint64_t* probs, const uint32_t* idx, uint64_t n, uint64_t* out,
                            cudaStream_t st);
// Terms idx[i] gathered; keys made natural with ctl->nat (ctl may be null:
// natural keys).
void launch_gather_terms(int prec, const uint32_t* idx, uint64_t n, const uint64_t* keys,
                         const void* amps, const uint64_t* probs, uint64_t* keys_out,
                         double* amps_out, uint64_t* probs_out, const Ctl* ctl, cudaStream_t st);
// Natural keys of stored keys (ctl->nat).
void launch_keys_natural(const uint64_t* keys, uint64_t n, const Ctl* ctl, uint64_t* out, cudaStream_t st);
// Load: amplitudes from double pairs (rounded to float for complex64),
// zeros dropped, duplicates flagged (input sorted by key); probabilities
// computed.  Count in ctl->count[2], duplicates in ctl->count[3].
void launch_load_compact(int prec, const uint64_t* sorted_keys, const uint32_t* idx, uint64_t n,
                         const double* amps_in, uint64_t* keys_out, void* amps_out,
                         uint64_t* probs_out, uint64_t* lookback, Ctl* ctl, cudaStream_t st);

}  // namespace sv
