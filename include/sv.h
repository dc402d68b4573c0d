/*
 * sv.h -- C ABI of the B300 sparse truncated state-vector library (libsv.so).
 *
 * The method (arXiv 2607.07816, "A Sparse and Truncated State Vector
 * Simulator for Peaked Circuits"):
 *   - the state stores only nonzero amplitudes, each with its basis state as a
 *     64-bit key (Sec. II, Sec. V); qubit i is bit i of the key; n <= 64
 *     (Sec. V);
 *   - a gate is a 2^m x 2^m unitary on m qubits applied to every group of
 *     basis states that differ only in those m bits (Eq. 3 and its
 *     generalisation in Sec. IV-A); contributions to one new basis state are
 *     summed (the segmented sum of Sec. IV-A) and exact zeros are dropped;
 *   - truncation keeps the largest-probability terms: p-mass first, then
 *     top-k, then renormalisation (Sec. III, Sec. IV-B);
 *   - the result read back is the most probable basis state (Sec. V).
 *
 * All compute runs in CUDA kernels on the handle's stream; the state stays
 * device-resident between calls.
 *
 * Conventions shared by every entry point:
 *   - Gate local index: r = sum_t bit(key, qubits[t]) << t (qubits[0] is the
 *     least significant bit).  U is row-major U[r_out][r_in], 2*4^m doubles
 *     interleaved (re, im).
 *   - Canonical order of terms: probability descending, then key ascending.
 *     prob = fma(re, re, im*im) in double (complex64 components widened).
 *   - Probability masses are exact sums of floor(prob * 2^120) held as
 *     128-bit integers, converted to double with round-to-nearest-even.
 *   - Ownership: every input buffer is read before the call returns; the
 *     caller may free it afterwards.  Output buffers belong to the caller.
 *   - Errors: every call returns an sv_status.  Arguments are validated on
 *     the host (SV_E_ARG).  Device-side failures (a bounded wait that ran
 *     out) are recorded on the handle and returned by the call that observes
 *     them; the handle then refuses further work with SV_E_STATE.
 *     sv_last_error() describes the last failure.
 *   - Threads: a handle must not be used by two host threads at once.
 */
#ifndef SV_H_
#define SV_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sv_state sv_state; /* opaque; owned by the caller until sv_destroy */

typedef enum {
  SV_OK = 0,
  SV_E_ARG = -1,          /* invalid argument (checked on the host) */
  SV_E_NOMEM = -2,        /* device allocation failed */
  SV_E_CUDA = -3,         /* a CUDA runtime call failed */
  SV_E_NOT_UNITARY = -4,  /* max |U^dagger U - I| above 1e-10 */
  SV_E_TIMEOUT = -5,      /* a bounded device-side wait ran out */
  SV_E_STATE = -6         /* handle unusable, or state empty / mass overflow */
} sv_status;

typedef enum { SV_C128 = 0, SV_C64 = 1 } sv_prec;

/* Device memory provider.  alloc returns device memory of at least `bytes`
 * bytes aligned to 256 bytes, or NULL on failure; free releases it.  A NULL
 * allocator pointer selects cudaMalloc / cudaFree. */
typedef struct {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* ctx;
} sv_allocator;

/* Create the state |0...0> (a single term, Sec. I) on n qubits (1..64),
 * complex128 amplitudes, the legacy default stream and cudaMalloc.
 * K >= 1 is the top-k limit, 0 < p <= 1 the p-mass threshold of Sec. III
 * (p >= 1 disables the p-mass cut). */
sv_status sv_create(int n, uint64_t K, double p, sv_state** out);

/* As sv_create with an amplitude precision (sv_prec), a cudaStream_t (NULL =
 * legacy default stream) and an allocator (NULL = cudaMalloc).  The first
 * handle created on a device sets the kernels' shared-memory limits there
 * (once per device; SV_E_CUDA if that fails).  A handle's calls must run
 * with the device it was created on current. */
sv_status sv_create_ex(int n, uint64_t K, double p, int prec, void* cuda_stream,
                       const sv_allocator* alloc, sv_state** out);

/* Size the handle's device buffers for states of up to `terms` terms and
 * the candidates of any gate on them (16 per term), so that later gates and
 * truncations allocate nothing (buffers otherwise grow, by doubling, when a
 * gate first needs more room; each growth allocates device memory, which
 * costs milliseconds per gigabyte).  Buffers never shrink.  About
 * terms * (16 * 2 * (16 + S) + 40) bytes with S the amplitude size (16 for
 * complex128, 8 for complex64).  SV_E_NOMEM when the device memory is not
 * there (the handle stays usable), SV_E_ARG above 2^32 - 1 terms.
 * Synchronises. */
sv_status sv_reserve(sv_state* s, uint64_t terms);

/* Free the handle and its device memory.  Accepts NULL. */
sv_status sv_destroy(sv_state* s);

/* Apply a 2^m x 2^m unitary (1 <= m <= 4) to the m distinct qubits
 * qubits[0..m-1] (Eq. 3, Sec. IV-A).  Never truncates.  U must be finite
 * and unitary within 1e-10 (SV_E_NOT_UNITARY otherwise).  Enqueued on the
 * handle's stream; the call waits for the new term count. */
sv_status sv_apply_gate(sv_state* s, int m, const int* qubits, const double* U);

/* Truncate by the rule of Sec. III: p-mass cut c_p (smallest prefix of the
 * canonical order whose mass reaches p * total), then c = min(c_p, K); if
 * c < N the first c terms are kept and scaled by 1/sqrt(kept mass).
 * kept (nullable) receives c; retained_fraction (nullable) receives
 * kept mass / total mass (1 when nothing was cut).  Waits for the cut; the
 * renormalising compaction is left running on the stream and the number of
 * terms it wrote is checked at the handle's next wait (an unexpected count
 * then fails that call with SV_E_STATE). */
sv_status sv_truncate(sv_state* s, uint64_t* kept, double* retained_fraction);

/* Most probable basis state in canonical order (Sec. V).  Synchronises;
 * 16 bytes come back to the host.  SV_E_STATE if the state is empty. */
sv_status sv_peak(sv_state* s, uint64_t* key, double* prob);

/* Pipelined form of sv_peak: enqueues the same readout on the handle's
 * stream together with a 16-byte copy into a pinned result slot and returns
 * at once with *ticket naming the result.  sv_peak_wait(s, ticket, ...)
 * then waits for that copy only (not for later work on the stream) and
 * returns the key and probability the state had when sv_peak_async was
 * called.  Eight results can be outstanding; a ticket older than the last
 * eight, or never issued, gives SV_E_ARG.  Device error flags are reported
 * by the handle's next waiting call.  SV_E_STATE if the state is empty. */
sv_status sv_peak_async(sv_state* s, uint64_t* ticket);
sv_status sv_peak_wait(sv_state* s, uint64_t ticket, uint64_t* key, double* prob);

/* Keys and probabilities in canonical order into host buffers of `cap`
 * entries; writes min(cap, N) entries and sets *count = N.  Either buffer
 * may be NULL.  Synchronises. */
sv_status sv_probs(sv_state* s, uint64_t* keys, double* probs, uint64_t cap, uint64_t* count);

/* Current number of terms. */
sv_status sv_num_terms(sv_state* s, uint64_t* N);

/* Product of the retained fractions of every truncation so far: the
 * fidelity estimate of Sec. III. */
sv_status sv_retained_mass(sv_state* s, double* F);

/* Keys and amplitudes (interleaved re, im as doubles) in canonical order
 * into host buffers of `cap` entries; writes min(cap, N), *count = N. */
sv_status sv_export(sv_state* s, uint64_t* keys, double* amps, uint64_t cap, uint64_t* count);

/* Replace the state with N host terms (checkpoint / test hook).  Keys must
 * be distinct and below 2^n (SV_E_ARG otherwise); zero amplitudes are not
 * stored; complex64 handles round each component to float. */
sv_status sv_load(sv_state* s, const uint64_t* keys, const double* amps, uint64_t N);

/* Primitives for one state held in several handles (one per GPU, each with
 * the terms of one partition of the basis states): the truncation of
 * Sec. III taken over the union of the handles' terms.  The canonical order
 * is that of the composite Z = (~prob_bits, natural key) read as a 128-bit
 * integer (ascending Z = probability descending, key ascending).
 *
 * sv_select_histogram: among this handle's terms whose Z agrees with
 * (prefix_hi, prefix_lo) on its top `bits` bits (0 <= bits <= 127), the
 * count and the exact fixed-point mass (floor(prob * 2^120) summed, as
 * hi, lo words) per value of the next D = min(11, 128 - bits) bits of Z:
 * counts[2048] and masses[2 * 2048] (bins >= 2^D stay zero).  Summed over
 * the handles, the levels of a radix select find the cut.  bits = 0 gives
 * the whole state's mass split by the top digit.  Synchronises. */
sv_status sv_select_histogram(sv_state* s, uint64_t prefix_hi, uint64_t prefix_lo, int bits, uint32_t* counts,
                              uint64_t* masses);

/* Keep this handle's terms whose Z is at most (z_hi, z_lo), in order, scaled
 * by 1 / sqrt(double(S_c)), and multiply the retained product by
 * double(S_c) / double(S_N), where S_c = (sc_hi, sc_lo) and
 * S_N = (sn_hi, sn_lo) are the kept and the total fixed-point masses of all
 * the handles together (the rule of sv_truncate, with the cut and the
 * masses decided across handles).  *kept (nullable) receives this handle's
 * terms left.  SV_E_ARG for a zero mass.  Synchronises. */
sv_status sv_cut(sv_state* s, uint64_t z_hi, uint64_t z_lo, uint64_t sc_hi, uint64_t sc_lo, uint64_t sn_hi,
                 uint64_t sn_lo, uint64_t* kept);

/* Human-readable description of the last failure on this handle (never
 * NULL; empty when there was none). */
const char* sv_last_error(const sv_state* s);

/* Statistics of the last sv_apply_gate / sv_truncate (for benchmarking):
 * terms before the gate, candidates after it, terms kept by the last
 * truncation, radix-sort passes run, select levels run, the total and kept
 * probability masses of the last truncation, how many of its selects ran on
 * the sampled window (window_hits) and the window size of the last one, and
 * how many gates so far were applied inside buckets of the state versus
 * through the global grouping sort. */
typedef struct {
  uint64_t n_in, n_pre, n_kept;
  uint32_t sort_passes;
  uint32_t select_levels;
  double total_mass, kept_mass;
  uint32_t window_hits;
  uint32_t selects;       /* select runs of the last truncation: top-k, then p-mass only when needed */
  uint64_t window_terms;
  uint64_t local_gates;   /* gates applied bucket-locally so far (no global sort) */
  uint64_t global_gates;  /* gates that needed the global sort so far */
  uint64_t local_fallbacks; /* local attempts redone globally (bucket too large) */
  uint64_t diag_gates;    /* gates applied in place as diagonal matrices so far */
  uint64_t mono_gates;    /* gates applied as permutations with phases (one output per term) so far */
} sv_stats;
sv_status sv_last_stats(const sv_state* s, sv_stats* out);

/* Phase timing for benchmarking.  With timing on, CUDA events recorded on
 * the handle's stream bracket each phase and the elapsed device times are
 * accumulated.  sv_set_timing also resets the accumulators.  Phases, in
 * order: 0 gate key transform + digit histograms, 1 radix-sort passes,
 * 2 partner-group heads, 3 group mat-vec, 4 truncation select levels,
 * 5 truncation compaction, 6 peak, 7 other (readout, load), 8 truncation
 * sample window pass, 9 bucket-local gate (and bucket-size check).  ms and
 * launches (nullable) receive SV_NUM_PHASES entries: milliseconds and kernel
 * launches.  sv_phase_times waits for the handle's stream first (with timing
 * on), so phases still in flight are included. */
#define SV_NUM_PHASES 10
sv_status sv_set_timing(sv_state* s, int enable);
sv_status sv_phase_times(const sv_state* s, double* ms, uint64_t* launches);

/* FP64 pipe throughput on the current device (benchmarking hook): one
 * launch of blocks_per_sm (1..32) blocks per SM, 256 threads each, every
 * thread running 8 independent fused multiply-add chains of `iters` steps
 * (no memory traffic), timed with CUDA events on the legacy default stream
 * after a shorter warm-up launch.  *tflops receives 2 flops per fma over the
 * elapsed time, *ms (nullable) the time.  SV_E_ARG for iters == 0 or a
 * blocks_per_sm outside 1..32. */
sv_status sv_probe_fp64(uint64_t iters, int blocks_per_sm, double* tflops, double* ms);

/* Gate application variant for the handle's next gates.  0 (default)
 * group-first -- bring every partner group together with the gate bits at
 * the bottom of the sort key, then expand each group to its 2^m outputs
 * inside the mat-vec (states of at most 4096 terms do all of it in shared
 * memory).  Every gate leaves the state sorted by its own sort key, and the
 * next gate's key keeps the other qubits in that order, so the grouping is
 * a stable partition by the gate bits followed by m levels of pairwise
 * merges.  2 group-first with the grouping done by a full LSD radix sort of
 * the sort keys (for comparison).  1 expand-first -- the paper's
 * formulation (Sec. IV-A): every term contributes one record to each of its
 * 2^m outputs, the records are sorted by (output, source gate bits) and each
 * output's contributions are summed in ascending source order.  All three
 * give the same terms and amplitudes bit for bit; expand-first sorts 2^m
 * times as many records and exists for comparison.  SV_E_ARG for other
 * values. */
sv_status sv_set_apply_variant(sv_state* s, int variant);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t sv_launch_count(void);

/* Bytes this library has moved host->device (copies and gate parameters)
 * and device->host (copies) in this process.  Either pointer may be NULL. */
void sv_transfer_bytes(uint64_t* h2d, uint64_t* d2h);

/* ---------------------------------------------------------------------
 * Batched form.  Many circuits share one device-resident state: each circuit
 * is a segment (a slot) with its own qubit count n (1..63) and top-k limit K.
 * One svb_step applies one gate to every listed slot (slots not listed are
 * left unchanged) and then truncates every slot above its K to its own top-K
 * (Sec. III, p-mass is not offered in this form).  All slots go through one
 * grouping sort, one mat-vec pass and one segmented select per step; each
 * slot's result is the one the single-state path gives for the same gates.
 * Gate conventions are those of sv_apply_gate.  Calls enqueue on the
 * handle's stream.  With one launch per step (the default, see
 * svb_set_layer_kernel) svb_step and svb_add return without waiting for
 * the device and svb_peak_async / svb_peak_wait read results pipelined;
 * the calls that report on a slot wait for the work enqueued before them.
 * With separate kernels every call synchronises before returning.
 * ------------------------------------------------------------------- */
typedef struct svb_state svb_state;
typedef struct {
  int slot;          /* target slot */
  int m;             /* 1..4 */
  int qubits[4];     /* qubits[0..m-1], distinct, below the slot's n */
  const double* U;   /* 2*4^m doubles, row-major U[r_out][r_in], (re, im); read before return */
} svb_gate;

/* Create a batch with room for max_slots (1..1023) circuits, amplitude
 * precision prec, a cudaStream_t (NULL: the handle creates a stream of its
 * own; every call returns when the work it needs is complete) and an
 * allocator (NULL = cudaMalloc). */
sv_status svb_create(int max_slots, int prec, void* cuda_stream, const sv_allocator* alloc, svb_state** out);
sv_status svb_destroy(svb_state* b);
/* Add a circuit in the state |0...0>; *slot receives its slot (the lowest
 * free one).  p must be 1 (top-k only).  One step sorts (slot, key) pairs as
 * 64-bit words, so the largest n among the slots in use plus the bits of the
 * highest slot index in use (floor(log2(top)) + 1, top = highest slot + 1,
 * counting slots removed since the last step) must stay within 64: n <= 54
 * always fits 1023 slots, n = 56 fits while at most 255 are in use.
 * SV_E_ARG when no slot is free or that bound would be broken (nothing
 * changes; the call can be retried after slots are retired). */
sv_status svb_add(svb_state* b, int n, uint64_t K, double p, int* slot);
/* Retire a slot; its terms are dropped by the next step and the slot is free
 * after it. */
sv_status svb_remove(svb_state* b, int slot);
/* One gate per listed slot (at most one per slot), then per-slot top-k. */
sv_status svb_step(svb_state* b, const svb_gate* gates, int count);
sv_status svb_num_terms(svb_state* b, int slot, uint64_t* N);
/* Product of the slot's retained fractions (Sec. III). */
sv_status svb_retained_mass(svb_state* b, int slot, double* F);
/* Most probable basis state of the slot in canonical order (Sec. V). */
sv_status svb_peak(svb_state* b, int slot, uint64_t* key, double* prob);
/* Pipelined readout of a slot: svb_peak_async enqueues the computation of
 * the slot's most probable basis state (as svb_peak) and its retained mass
 * on the handle's stream behind the steps enqueued so far, and returns a
 * ticket at once; svb_peak_wait(ticket) waits for that readout only and
 * returns its results (F may be NULL).  The slot may be removed right after
 * svb_peak_async.  At most 1024 readouts can be outstanding (SV_E_STATE
 * beyond); each ticket is collected once.  With one launch per step the
 * steps themselves do not wait either, so a serving loop can enqueue the
 * next step before it collects the readouts of the last one. */
sv_status svb_peak_async(svb_state* b, int slot, uint64_t* ticket);
sv_status svb_peak_wait(svb_state* b, uint64_t ticket, uint64_t* key, double* prob, double* F);
/* The slot's keys and amplitudes (interleaved re, im doubles) in storage
 * order, min(cap, N) of them; *count = N. */
sv_status svb_export(svb_state* b, int slot, uint64_t* keys, double* amps, uint64_t cap, uint64_t* count);
const char* svb_last_error(const svb_state* b);
/* Autotuning of the step's launch shapes (on by default): for every class of
 * step (kernel, precision, widest gate of the step, floor(log2) of the term
 * count) each candidate shape is timed twice on live steps with CUDA events,
 * then the fastest is kept: with one launch per step, the layer kernel's
 * blocks per SM (the most that fit, or one fewer; classes by the term count
 * in factors of 4; a launch's time is read once the step after next reuses
 * its table set, so tuning adds no wait); with separate kernels, the group mat-vec's groups per thread and the
 * select scan's and the compaction's blocks per SM.  Every shape computes the
 * same result.  Off: fixed default shapes. */
sv_status svb_set_autotune(svb_state* b, int on);
/* Timed trials so far, step classes seen, and classes whose every shape has
 * been timed (the tuner has settled them). */
sv_status svb_autotune_stats(const svb_state* b, uint64_t* trials, uint64_t* classes, uint64_t* settled);
/* CUDA graphs (on by default): once a step's launch shapes are settled, each
 * of its two enqueued parts (gate table upload through the first select
 * levels; compaction and read-back) is captured into a graph the first time
 * its sizes, shapes and buffers occur, and replayed when they recur (steps
 * of circuits at their K repeat exactly).  Off: direct launches.  Results
 * are the same either way. */
sv_status svb_set_graphs(svb_state* b, int on);
/* Graphs captured and graph launches so far. */
sv_status svb_graph_stats(const svb_state* b, uint64_t* captures, uint64_t* launches);
/* One launch per step (on by default): the whole step (sort keys, grouping,
 * group heads, mat-vec, per-slot top-k select to the exact cut,
 * renormalising compaction) runs as one persistent cooperative kernel whose
 * blocks pass grid-wide barriers between the phases, with every size read
 * on the device.  With graphs on, the gate-table upload and the launch are
 * one graph, captured when the step's table size, widest gate and buffers
 * recur and replayed after that.  The device then keeps the state's term
 * count, slot ranges and retained masses, svb_step and svb_add return
 * without waiting, and the calls that report on a slot (svb_num_terms,
 * svb_retained_mass, svb_peak, svb_export) wait for the steps enqueued
 * before them; device errors of a step are returned by the next call that
 * waits.  Off: the step's separate kernels (two parts, a host wait after
 * each, autotuned launch shapes).  Results are the same either way.  Only
 * an empty batch changes mode (SV_E_STATE otherwise). */
sv_status svb_set_layer_kernel(svb_state* b, int on);
/* Benchmarking hook: milliseconds spent in each phase of the one-launch
 * step, summed over the handle's steps, as timed by the kernel's first block
 * from one grid barrier to the next (setup, sort keys, partition counts,
 * partition offsets, partition scatter, merge splits, merge levels, group
 * heads, mat-vec, select state, first pick, select scans, picks, finishes,
 * scales, compaction).  Writes min(cap, *count) values; *count = the number
 * of phases. */
sv_status svb_layer_phase_times(svb_state* b, double* ms, int cap, int* count);

/* Peak readout that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc where they need
 * the readout (their device memory is owned by another runtime or pool,
 * they run under a fixed device-memory budget, or an allocation would stall
 * the device at that point).  The caller passes its own device arrays:
 * keys[n] (uint64) and amps[n] (double2 for SV_C128, float2 for SV_C64),
 * a cudaStream_t (NULL = legacy default stream), and host outputs for the
 * most probable key and its probability (canonical order: probability
 * descending, key ascending).  Working memory is a fixed 64 KiB + 256 B
 * array inside the library, so 1 <= n <= 2^28 (SV_E_ARG otherwise).  The
 * first call on a device looks up that array's device address; make it
 * before any stream capture.  All calls on a device share the array: calls
 * that overlap on the GPU race.  Synchronises the stream. */
sv_status sv_peak_noalloc(int prec, const uint64_t* keys, const void* amps, uint64_t n,
                          void* cuda_stream, uint64_t* key, double* prob);

/* Device self-test of the complex64 arithmetic that the library forms
 * without float<->double conversion instructions (widening and rounding by
 * bit manipulation, bit-identical by construction): which = 0 checks the
 * probability fma(double(re), double(re), double(im) * double(im)),
 * which = 1 the rescaled amplitude float(double(x) * s).  n cases drawn from
 * seed (random bit patterns, subnormals, few-bit significands for exact
 * rounding ties) are compared on the default stream with the results of the
 * conversion instructions; *mismatches receives the count and *first_bad
 * the lowest failing case index (UINT64_MAX when none).  which = 2 checks
 * the bounded waits of the library's scans instead: a kernel waits for a
 * descriptor that nothing publishes, must give up after its poll limit and
 * flag a timeout, and return normally (the CUDA context stays usable);
 * *mismatches is 0 when it did, and *first_bad receives the error flags it
 * raised.  SV_E_ARG for another `which` or NULL outputs. */
sv_status sv_selftest(int which, uint64_t n, uint64_t seed, uint64_t* mismatches, uint64_t* first_bad);

#ifdef __cplusplus
}
#endif
#endif /* SV_H_ */
