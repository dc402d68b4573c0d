// Internal interfaces of the batched (segmented) form.
#pragma once

#include "internal.h"

namespace sv {

// Gate of one segment for one step.  m == 0 is the identity (each term its
// own group); m < 0 marks a removed segment whose terms are dropped.
//
// Segments are contiguous in the buffer, in the order of their ranks (new
// circuits are appended at the end); the sort key's segment field is the
// rank, and rank_slot maps it back to the slot.
//
// Keys stay natural (qubit i = bit i), but each segment is kept sorted by a
// sort order of its own that evolves as in the single-state path: a gate's
// sort key puts its qubits at the bottom (qubits[t] at bit t) and keeps the
// other qubits in the order of the previous sort key.  pos[b] is the bit of
// qubit b in this step's sort key.  Because the segment is sorted by the
// previous order, its terms with equal gate bits are already in the new
// order, so the batch is grouped by a stable partition and merges.
struct SegGate {
  uint64_t K;  // top-k limit of the slot (0: slot not in use)
  int m;
  int q[4];   // gate order (bit t of r)
  int qs[4];  // the same qubits ascending
  uint32_t re_nz[16];
  uint32_t im_nz[16];
  uint32_t rank;  // the segment's place in the buffer (the sort key's segment field)
  uint8_t pos[64];
  double U[512];
};

// Per-slot nibble tables of this step's sort order: fwd maps a natural key
// to its sort key, inv a sort key back to the natural key (16 x 16 words
// each, fwd first).
constexpr int SEG_TABLE_WORDS = 2 * 16 * 16;

__device__ __forceinline__ uint32_t seg_gather_r(uint64_t key, const int* q, int m) {
  uint32_t r = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (t < m) r |= (uint32_t)((key >> q[t]) & 1ull) << t;
  return r;
}

__device__ __forceinline__ uint64_t seg_deposit_r(uint32_t r, const int* q, int m) {
  uint64_t x = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (t < m) x |= (uint64_t)((r >> t) & 1u) << q[t];
  return x;
}

// Select state of one segment (top-k by count, as the single-state select).
struct SegSel {
  uint32_t active;     // this segment is truncated in this step
  uint32_t done;       // 1: cut found, 2: no cut
  uint32_t bits;
  uint32_t pad;
  uint64_t prefix_hi, prefix_lo;
  uint64_t target;     // rank of the cut (K)
  uint64_t before_count;
  uint64_t before_mass_hi, before_mass_lo;
  uint64_t bin_count;
  uint64_t total_mass_hi, total_mass_lo;
  uint64_t cut_pbits, cut_key, cut_count;
  uint64_t cut_mass_hi, cut_mass_lo;
  double scale;
};

// ---------------------------------------------------------------- one launch per layer
// Per-step scalars of the layer kernel, uploaded with the gate table (so a
// captured launch reads the current step's values).
struct LayerStep {
  int shift;  // bit of the segment rank in the sort key
  int top;    // slots in the gate table
  int m;      // grouping width: the widest gate of the step, at least 1
  int pad;
};

// Phases of the layer kernel, as timed by its first block (the time from
// one grid barrier to the next: the slowest block's work plus the barrier).
enum LayerPhase {
  LP_SETUP, LP_KEYS, LP_COUNTS, LP_OFFSETS, LP_SCATTER, LP_SPLITS, LP_MERGE, LP_HEADS, LP_APPLY, LP_INIT,
  LP_PICK1, LP_HIST, LP_PICK, LP_FINISH, LP_SCALE, LP_TRUNC, LP_COUNT
};

// Control words of the layer kernel (zeroed when the handle is created).
// With one launch per step the device holds the state's bookkeeping: which
// of the two buffer sets holds the state, its term count, the slot bounds
// (in bounds[0..1] after a step without a cut, bounds[2..3] after one) and
// every slot's retained mass; the host reads them when it needs them.
struct LayerCtl {
  uint32_t bar_count, bar_gen;  // grid barrier
  uint32_t truncated;           // 1: the last step cut a slot (its bounds are the second pair)
  uint32_t unresolved;          // 1: a slot's cut was not found within LAYER_LEVELS select levels
  uint32_t cur;                 // buffer set holding the state
  uint32_t pad;
  uint64_t n_cur;               // terms in the state
  uint64_t t_last;              // global timer at the last barrier (first block)
  uint64_t phase_ns[LP_COUNT];  // time per phase, summed over the steps
};

// Buffers of one layer launch.  The state moves from the input buffers to
// the mat-vec buffers and, when a slot is cut, to the truncation buffers
// (the input buffers again: the input is dead once the mat-vec has run).
struct LayerParams {
  const LayerStep* step;
  LayerCtl* lc;
  Ctl* ctl;
  uint64_t* keys[2];  // the two buffer sets: the state in lc->cur, the mat-vec output in the other,
  void* amps[2];      // a compaction back into lc->cur
  uint64_t* probs[2];
  uint16_t* seg[2];
  double* F;          // [slots] retained mass of every slot
  uint64_t* sk[2];
  uint32_t* sidx[2];
  uint32_t* heads;
  uint32_t* hist16;
  uint32_t* part;  // partition counts and offsets (2 * 16 * tiles words), then merge splits
  uint64_t* lb;    // look-back words: heads, mat-vec and compaction regions in turn
  uint64_t lb_heads_words, lb_apply_words, lb_trunc_words;
  const SegGate* gates;
  const uint16_t* rank_slot;
  uint64_t* tables;
  SegSel* sel;
  uint32_t* sel_cnt[2];   // [slots][SEL_BINS] each (two parities: one level reads, the next clears)
  uint64_t* sel_mass[2];  // [slots][4] each
  uint64_t* sel_buf;
  uint32_t* sel_bufn[2];  // [slots] each
  uint64_t* start;  // slot bounds in the mat-vec output (start all ones for a slot with no terms)
  uint64_t* end;
  uint64_t* start_tr;  // slot bounds after the compaction
  uint64_t* end_tr;
};

// Append the state |0> of a new slot at the end of the device-held state
// (layer bookkeeping: lc->n_cur grows by one, the slot's bounds and retained
// mass are set).
void launch_seg_append_layer(uint64_t* const keys[2], void* const amps[2], uint64_t* const probs[2],
                             uint16_t* const seg[2], LayerCtl* lc, uint64_t* bounds, int max_slots, double* F,
                             int slot, int prec, cudaStream_t st);
// Peak of one slot (canonical order over its amplitudes' probabilities) into
// out = {key, probability bits, retained mass bits}: with dev_range the
// slot's range, buffer set and mass come from the layer bookkeeping, else
// from (off, count, cur) and F_host.  part: [PEAK_SEG_BLOCKS][2] scratch.
constexpr int PEAK_SEG_BLOCKS = 148 * 2;
void launch_seg_peak(uint64_t* const keys[2], void* const amps[2], int prec, int dev_range, const LayerCtl* lc,
                     const uint64_t* bounds, int max_slots, const double* F, int slot, uint64_t off, uint64_t count,
                     int cur, double F_host, uint64_t* part, uint64_t* out, cudaStream_t st);

// Blocks of one cooperative layer launch on this device (all co-resident).
cudaError_t seg_layer_grid(int prec, int m, int sms, unsigned* grid);
// Enqueue the layer kernel (cooperative launch of `grid` blocks).
cudaError_t launch_seg_layer(int prec, int m, const LayerParams& P, unsigned grid, cudaStream_t st);

cudaError_t batch_prepare();  // kernel attributes of this device, before any stream capture
void launch_seg_tables(const SegGate* gates, int slots, uint64_t* tables, cudaStream_t st);
void launch_seg_keys(const uint64_t* keys, const uint16_t* seg, uint64_t n, const SegGate* gates,
                     const uint64_t* tables, int shift, uint64_t* sk, cudaStream_t st);
void launch_seg_heads(const uint64_t* sk, uint64_t n, int shift, const SegGate* gates, const uint16_t* rank_slot,
                      uint32_t* heads,
                      uint64_t* lookback, Ctl* ctl, cudaStream_t st);
// Launch shapes that the batched step tunes (every shape gives the same
// result): the mat-vec's groups per thread, the select scan's and the
// compaction's blocks per SM.
int seg_apply_configs(int mmax);
constexpr int SEGSEL_CONFIGS = 3;
constexpr int SEGTRUNC_CONFIGS = 2;
void launch_seg_apply(int prec, const uint64_t* sk, const uint32_t* sidx, uint64_t n, const uint32_t* heads,
                      const void* amps_in, int shift, int mmax, const SegGate* gates, const uint16_t* rank_slot,
                      const uint64_t* keys_in, uint64_t* keys_out,
                      void* amps_out, uint64_t* probs_out, uint16_t* seg_out, uint32_t* hist1, uint64_t* start,
                      uint64_t* end, uint64_t* lookback, Ctl* ctl, uint64_t max_tiles, int cfg, cudaStream_t st);
// Sizes marked n_dev are read on the device (a term count written by an
// earlier kernel on the stream); launches are sized for at most n_max terms.
void launch_segsel_init(SegSel* sel, const SegGate* gates, const uint64_t* start, const uint64_t* end, int slots,
                        cudaStream_t st);
constexpr int SEGSEL_CAP = 4096;  // terms per segment copied for the finish kernel
void launch_segsel_level(const uint64_t* probs, const uint64_t* keys, const uint16_t* seg, const uint64_t* n_dev,
                         SegSel* sel, int slots, uint32_t* g_cnt, uint64_t* g_sum, uint64_t* g_buf, uint32_t* g_bufn,
                         uint32_t* err, int cfg, cudaStream_t st);
// The first level's pick from the histogram the mat-vec counted (hist1).
void launch_segsel_pick(SegSel* sel, int slots, const uint32_t* g_cnt, cudaStream_t st);
void launch_segsel_finish(const uint64_t* g_buf, const uint32_t* g_bufn, const uint64_t* g_sum, SegSel* sel,
                          int slots, uint32_t* err, cudaStream_t st);
void launch_segsel_scale(SegSel* sel, int slots, cudaStream_t st);
// The compaction writes keys, amplitudes and slots; the probabilities of
// the kept terms are not written (the next mat-vec computes its own, and a
// readout first recomputes them with launch_amp_probs).
void launch_seg_truncate(int prec, const uint64_t* keys, const void* amps, const uint64_t* probs, const uint16_t* seg,
                         const uint64_t* n_dev, uint64_t n_max, const SegSel* sel, uint64_t* keys_out,
                         void* amps_out, uint16_t* seg_out, uint64_t* start, uint64_t* end, uint64_t* lookback,
                         Ctl* ctl, int cfg, cudaStream_t st);
void launch_seg_append(uint64_t* keys, void* amps, uint64_t* probs, uint16_t* seg, uint64_t at, int slot, int prec,
                       cudaStream_t st);

}  // namespace sv
