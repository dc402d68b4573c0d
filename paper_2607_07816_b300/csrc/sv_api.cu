// C ABI of libsv.so (declared in include/sv.h): the state engine that
// sequences the kernels of one gate application, one truncation and the
// readouts on the handle's stream.
//
// Per gate (Sec. IV-A): grouping of the terms by the gate's sort key (the
// qubits outside the gate in the state's current order, the gate bits at the
// bottom) by a stable partition on the gate bits and pairwise merges ->
// partner-group heads with their output positions -> per-group mat-vec,
// exact zeros removed by an order-preserving pass when there are any; states
// of at most 4096 terms do the gate in one shared-memory kernel.
// Per truncation (Sec. III, Sec. IV-B): sampled window, radix select of the
// cut on the canonical composite by mass (p) and/or by count (K) ->
// renormalising compaction.  Readout (Sec. V): argmax in canonical order.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "host_util.h"
#include "internal.h"
#include "sv.h"

using namespace sv;

// Phases timed with CUDA events when timing is on (sv_set_timing).
enum Phase { PH_KEYS = 0, PH_SORT, PH_HEADS, PH_APPLY, PH_SELECT, PH_COMPACT, PH_PEAK, PH_OTHER, PH_WINDOW, PH_LOCAL, PH_COUNT };

static std::atomic<uint64_t> g_launches{0};
static std::atomic<uint64_t> g_h2d{0}, g_d2h{0};  // bytes crossing PCIe (copies and gate parameters)

struct sv_state {
  int n = 0;
  uint64_t K = 0;
  double p = 1.0;
  int prec = 0;
  cudaStream_t st = nullptr;
  sv_allocator alloc{};
  bool custom_alloc = false;
  size_t amp_bytes = 16;

  uint64_t N = 0;
  uint64_t cap = 0;
  uint64_t* keys[2] = {nullptr, nullptr};
  void* amps[2] = {nullptr, nullptr};
  uint64_t* probs[2] = {nullptr, nullptr};
  int cur = 0;

  uint64_t sort_cap = 0;
  uint64_t* sk[2] = {nullptr, nullptr};
  uint32_t* sidx[2] = {nullptr, nullptr};
  uint32_t* heads = nullptr;
  uint32_t* gmask = nullptr;  // per group: present mask | output mask << 16
  uint64_t* ooff = nullptr;   // per group: first output position
  uint64_t lb_entries = 0;
  uint64_t* lookback = nullptr;
  uint64_t gs_lb_entries = 0;
  uint64_t* gs_lb = nullptr;  // the group scan's two look-backs (cleared with the gate's tables)

  uint32_t* hist = nullptr;
  uint32_t* hist_host = nullptr;
  uint64_t* tile_counter = nullptr;
  SelectScratch ss{};
  Ctl* ctl = nullptr;
  Ctl* ctl_host = nullptr;

  double F = 1.0;
  std::string err;
  bool broken = false;
  sv_stats stats{};

  // 0: group-first, grouping by partition and merge; 1: expand-first;
  // 2: group-first, grouping by a full radix sort
  int variant = 0;
  // order[b]: bit of qubit b in the sort key the state is sorted by (every
  // gate leaves the state in its own sort-key order); order_next: the order
  // the gate being applied will leave
  int order[64] = {};
  int order_next[64] = {};
  // a truncation returns without waiting for its compaction; the count it
  // wrote is compared with the cut at the next wait on the stream
  bool kept_pending = false;
  uint64_t kept_expected = 0;
  // per-block best kept terms of the last compaction; valid until the state
  // changes again (the peak readout then reduces them)
  uint64_t* peak_part = nullptr;
  uint32_t peak_blocks = 0;
  bool peak_ready = false;
  bool probs_valid = true;  // probs[cur] holds every term's probability (a compaction leaves them stale)
  // pipelined peak readouts: results copied into a ring of pinned slots,
  // each with the event that marks its copy done
  static constexpr uint32_t PEAK_RING = 8;
  uint64_t* peak_host = nullptr;  // [PEAK_RING][2] (probability bits, key)
  cudaEvent_t peak_ev[PEAK_RING] = {};
  uint64_t peak_issued = 0;
  // the complex128 mat-vec left the exact total mass of the current terms in
  // ctl->total_mass (valid until the terms change)
  bool total_ready = false;
  int64_t gate_index = 0;
  GateTables* tab_dev = nullptr;   // this gate's permutation and U
  GateTables* tab_host = nullptr;  // pinned staging of tab_dev
  uint64_t local_gates = 0, global_gates = 0, local_fallbacks = 0;

  bool timing = false;
  cudaEvent_t ev_beg[PH_COUNT] = {};
  cudaEvent_t ev_end[PH_COUNT] = {};
  bool ph_pending[PH_COUNT] = {};
  double ph_ms[PH_COUNT] = {};
  uint64_t ph_launches[PH_COUNT] = {};
};

namespace {

constexpr uint64_t MAX_TERMS = (1ull << 32) - 1;  // 32-bit term indices in the sort payload

void* dev_alloc(sv_state* s, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (s->custom_alloc) return s->alloc.alloc(bytes, s->alloc.ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(sv_state* s, void* p) {
  if (!p) return;
  if (s->custom_alloc) {
    cudaStreamSynchronize(s->st);  // work enqueued without a wait may still use p
    s->alloc.free(p, s->alloc.ctx);
  } else {
    cudaFree(p);
  }
}

void ph_begin(sv_state* s, int ph) {
  if (s->timing) cudaEventRecord(s->ev_beg[ph], s->st);
}

void ph_end(sv_state* s, int ph) {
  if (s->timing) {
    cudaEventRecord(s->ev_end[ph], s->st);
    s->ph_pending[ph] = true;
  }
}

// After a stream synchronisation: fold finished phase intervals in.
void ph_collect(sv_state* s) {
  if (!s->timing) return;
  for (int ph = 0; ph < PH_COUNT; ++ph) {
    if (!s->ph_pending[ph]) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->ev_beg[ph], s->ev_end[ph]) == cudaSuccess) s->ph_ms[ph] += ms;
    s->ph_pending[ph] = false;
  }
  cudaGetLastError();
}

void launched(sv_state* s, int ph, uint64_t k) {
  s->ph_launches[ph] += k;
  g_launches += k;
}

sv_status fail(sv_state* s, sv_status code, const std::string& msg) {
  s->err = msg;
  return code;
}

sv_status cuda_check(sv_state* s, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return SV_OK;
  s->broken = true;
  return fail(s, SV_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Wait for the stream and read the control block; device error bits make
// the handle unusable.
sv_status sync_ctl(sv_state* s, const char* where) {
  cudaError_t e = cudaMemcpyAsync(s->ctl_host, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->st);
  g_d2h += sizeof(Ctl);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  sv_status rc = cuda_check(s, e, where);
  if (rc != SV_OK) return rc;
  ph_collect(s);
  if (s->ctl_host->err & ERR_TIMEOUT) {
    s->broken = true;
    return fail(s, SV_E_TIMEOUT, std::string(where) + ": a bounded device wait ran out");
  }
  if (s->ctl_host->err & ERR_INVARIANT) {
    s->broken = true;
    return fail(s, SV_E_STATE, std::string(where) + ": duplicate keys in the state");
  }
  if (s->kept_pending) {
    s->kept_pending = false;
    if (s->ctl_host->kept_check != s->kept_expected) {
      s->broken = true;
      return fail(s, SV_E_STATE, std::string(where) + ": truncation kept an unexpected number of terms");
    }
  }
  if (s->ctl_host->err & ERR_MASS) {
    s->broken = true;
    return fail(s, SV_E_STATE, std::string(where) + ": probability mass out of fixed-point range");
  }
  return SV_OK;
}

sv_status ensure_lookback(sv_state* s, uint64_t entries) {
  if (entries <= s->lb_entries) return SV_OK;
  uint64_t want = entries + entries / 2 + 1024;
  uint64_t* p = (uint64_t*)dev_alloc(s, want * sizeof(uint64_t));
  if (!p) return fail(s, SV_E_NOMEM, "look-back buffer allocation failed");
  dev_free(s, s->lookback);
  s->lookback = p;
  s->lb_entries = want;
  return SV_OK;
}

// State buffers (both halves) hold at least `need` terms; the current
// state is preserved.
sv_status ensure_state_cap(sv_state* s, uint64_t need) {
  if (need <= s->cap) return SV_OK;
  uint64_t cap = s->cap * 2 > need ? s->cap * 2 : need;
  if (cap < 4096) cap = 4096;
  uint64_t* k[2];
  void* a[2];
  uint64_t* pr[2];
  for (int i = 0; i < 2; ++i) {
    k[i] = (uint64_t*)dev_alloc(s, cap * 8);
    a[i] = dev_alloc(s, cap * s->amp_bytes);
    pr[i] = (uint64_t*)dev_alloc(s, cap * 8);
    if (!k[i] || !a[i] || !pr[i]) {
      for (int j = 0; j <= i; ++j) {
        dev_free(s, k[j]);
        dev_free(s, a[j]);
        dev_free(s, pr[j]);
      }
      return fail(s, SV_E_NOMEM, "state buffer allocation failed");
    }
  }
  if (s->N) {
    cudaMemcpyAsync(k[0], s->keys[s->cur], s->N * 8, cudaMemcpyDeviceToDevice, s->st);
    cudaMemcpyAsync(a[0], s->amps[s->cur], s->N * s->amp_bytes, cudaMemcpyDeviceToDevice, s->st);
    cudaMemcpyAsync(pr[0], s->probs[s->cur], s->N * 8, cudaMemcpyDeviceToDevice, s->st);
  }
  sv_status rc = cuda_check(s, cudaStreamSynchronize(s->st), "state growth");
  for (int i = 0; i < 2; ++i) {
    dev_free(s, s->keys[i]);
    dev_free(s, s->amps[i]);
    dev_free(s, s->probs[i]);
    s->keys[i] = k[i];
    s->amps[i] = a[i];
    s->probs[i] = pr[i];
  }
  s->cur = 0;
  s->cap = cap;
  return rc;
}

sv_status ensure_gs_lb(sv_state* s, uint64_t words) {
  if (words <= s->gs_lb_entries) return SV_OK;
  dev_free(s, s->gs_lb);
  s->gs_lb_entries = 0;
  s->gs_lb = (uint64_t*)dev_alloc(s, (words + words / 2) * sizeof(uint64_t));
  if (!s->gs_lb) return fail(s, SV_E_NOMEM, "group scan look-back allocation failed");
  s->gs_lb_entries = words + words / 2;
  return SV_OK;
}

sv_status ensure_sort_cap(sv_state* s, uint64_t need) {
  if (need > s->sort_cap) {
    uint64_t cap = s->sort_cap * 2 > need ? s->sort_cap * 2 : need;
    if (cap < 4096) cap = 4096;
    for (int i = 0; i < 2; ++i) {
      dev_free(s, s->sk[i]);
      dev_free(s, s->sidx[i]);
      s->sk[i] = (uint64_t*)dev_alloc(s, cap * 8);
      s->sidx[i] = (uint32_t*)dev_alloc(s, cap * 4);
    }
    dev_free(s, s->heads);
    dev_free(s, s->gmask);
    dev_free(s, s->ooff);
    s->heads = (uint32_t*)dev_alloc(s, cap * 4);
    s->gmask = (uint32_t*)dev_alloc(s, cap * 4);
    s->ooff = (uint64_t*)dev_alloc(s, cap * 8);
    if (!s->sk[0] || !s->sk[1] || !s->sidx[0] || !s->sidx[1] || !s->heads || !s->gmask || !s->ooff) {
      s->sort_cap = 0;
      return fail(s, SV_E_NOMEM, "sort buffer allocation failed");
    }
    s->sort_cap = cap;
  }
  return ensure_lookback(s, sort_tiles(need) * RADIX + 16);
}

SortScratch sort_scratch(sv_state* s) {
  SortScratch sc;
  sc.hist = s->hist;
  sc.hist_host = s->hist_host;
  sc.lookback = s->lookback;
  sc.lookback_tiles = s->lb_entries / RADIX;
  sc.tile_counter = s->tile_counter;
  sc.err = &s->ctl->err;
  return sc;
}

// Sort (sk[0], sidx[0]) on nbits bits; histograms are computed first unless
// hist_ready.  Returns the buffer index holding the result.
sv_status sort_pairs(sv_state* s, uint64_t n, int nbits, bool hist_ready, int* which, int* passes) {
  if (!hist_ready) {
    launch_digit_hist(s->sk[0], n, nbits, s->hist, s->st);
    launched(s, PH_OTHER, n ? 1 : 0);
  }
  cudaMemcpyAsync(s->hist_host, s->hist, sizeof(uint32_t) * MAX_PASSES * RADIX, cudaMemcpyDeviceToHost,
                  s->st);
  g_d2h += sizeof(uint32_t) * MAX_PASSES * RADIX;
  sv_status rc = cuda_check(s, cudaStreamSynchronize(s->st), "digit histogram");
  if (rc != SV_OK) return rc;
  ph_collect(s);
  cudaError_t e;
  ph_begin(s, PH_SORT);
  *which = radix_sort_pairs(s->sk[0], s->sidx[0], s->sk[1], s->sidx[1], n, nbits, sort_scratch(s),
                            s->st, passes, &e);
  ph_end(s, PH_SORT);
  launched(s, PH_SORT, (uint64_t)*passes);
  return cuda_check(s, e, "radix sort");
}

// Keys-only sort of s->sk[0] on the bits [lo, lo + nbits) (the histograms of
// those digits are already in s->hist).
sv_status sort_keys(sv_state* s, uint64_t n, int lo, int nbits, int* which, int* passes) {
  cudaMemcpyAsync(s->hist_host, s->hist, sizeof(uint32_t) * MAX_PASSES * RADIX, cudaMemcpyDeviceToHost,
                  s->st);
  g_d2h += sizeof(uint32_t) * MAX_PASSES * RADIX;
  sv_status rc = cuda_check(s, cudaStreamSynchronize(s->st), "digit histogram");
  if (rc != SV_OK) return rc;
  ph_collect(s);
  cudaError_t e;
  ph_begin(s, PH_SORT);
  *which = radix_sort_keys(s->sk[0], s->sk[1], n, lo, nbits, sort_scratch(s), s->st, passes, &e);
  ph_end(s, PH_SORT);
  launched(s, PH_SORT, (uint64_t)*passes);
  return cuda_check(s, e, "radix sort");
}

// The state's probabilities, recomputed from its amplitudes when a
// compaction left them stale (the compactions rescale the kept terms but
// compute new probabilities only for the peak candidates).
void ensure_probs(sv_state* s) {
  if (s->probs_valid) return;
  launch_amp_probs(s->prec, s->amps[s->cur], s->N, s->probs[s->cur], s->st);
  launched(s, PH_OTHER, 1);
  s->probs_valid = true;
}

// Canonical order (probability descending, key ascending) of the current
// state: the permutation ends in sidx[*which].
sv_status canonical_perm(sv_state* s, int* which) {
  uint64_t N = s->N;
  ensure_probs(s);
  sv_status rc = ensure_sort_cap(s, N);
  if (rc != SV_OK) return rc;
  launch_iota(s->sidx[0], N, s->st);
  launch_keys_natural(s->keys[s->cur], N, s->ctl, s->sk[0], s->st);  // the stored keys in qubit order
  launched(s, PH_OTHER, 2);
  int w = 0, passes = 0;
  rc = sort_pairs(s, N, s->n, false, &w, &passes);
  if (rc != SV_OK) return rc;
  // second, stable sort by ~prob_bits (ascending = probability descending)
  launch_not_bits_gather(s->probs[s->cur], s->sidx[w], N, s->sk[1 - w], s->st);
  launch_digit_hist(s->sk[1 - w], N, 63, s->hist, s->st);
  launched(s, PH_OTHER, 2);
  cudaMemcpyAsync(s->hist_host, s->hist, sizeof(uint32_t) * MAX_PASSES * RADIX, cudaMemcpyDeviceToHost,
                  s->st);
  rc = cuda_check(s, cudaStreamSynchronize(s->st), "digit histogram");
  if (rc != SV_OK) return rc;
  cudaError_t e;
  int w2 = radix_sort_pairs(s->sk[1 - w], s->sidx[w], s->sk[w], s->sidx[1 - w], N, 63,
                            sort_scratch(s), s->st, &passes, &e);
  launched(s, PH_OTHER, (uint64_t)passes);
  rc = cuda_check(s, e, "radix sort");
  if (rc != SV_OK) return rc;
  // radix_sort_pairs returns 0 for (kA, vA) = (sk[1-w], sidx[w]) and 1 for (sk[w], sidx[1-w])
  *which = (w2 == 0) ? w : 1 - w;
  return SV_OK;
}




// The natural-key table of the state's current order (after create and
// load, when no gate has set it).
sv_status upload_nat(sv_state* s) {
  build_nat_table(s->n, s->order, s->tab_host->nat);
  const size_t bytes = offsetof(GateTables, U);
  g_h2d += sizeof(s->tab_host->nat);
  launch_store_tables(*s->tab_host, s->tab_dev, bytes, GateReset{nullptr, nullptr, nullptr, 0}, s->st);
  launched(s, PH_OTHER, 1);
  return cuda_check(s, cudaGetLastError(), "natural-key table upload");
}

// Sort-key permutation of the gate for the state's current order, uploaded
// for the kernels; the order it leaves goes to order_next.
sv_status upload_perm(sv_state* s, GateParams& gp, const GateReset& reset = GateReset{nullptr, nullptr, nullptr, 0}) {
  build_gate_tables(s->n, gp.m, gp.q, s->order, s->tab_host, gp.qpos, s->order_next);
  gp.perm = &s->tab_dev->perm;
  gp.U = s->tab_dev->U;
  gp.n = s->n;
  gp.tbits = 0;
  gp.pmask = 0;
  // the permutation, the natural-key table and the 2 d^2 doubles of U travel
  // as the parameters of one small kernel that stores them (no copy-engine
  // transfer to wait for in the stream)
  const size_t bytes = offsetof(GateTables, U) + sizeof(double) * 2 * (1u << (2 * gp.m));
  g_h2d += bytes;
  launch_store_tables(*s->tab_host, s->tab_dev, bytes, reset, s->st);
  launched(s, PH_OTHER, 1);
  return cuda_check(s, cudaGetLastError(), "gate table upload");
}

#define SV_GUARD(s)                                                    \
  do {                                                                 \
    if (!(s)) return SV_E_ARG;                                         \
    if ((s)->broken) return fail((s), SV_E_STATE, "handle unusable after an earlier failure: " + (s)->err); \
  } while (0)

}  // namespace

extern "C" {

sv_status sv_create_ex(int n, uint64_t K, double p, int prec, void* cuda_stream,
                       const sv_allocator* alloc, sv_state** out) {
  if (!out) return SV_E_ARG;
  *out = nullptr;
  if (n < 1 || n > 64 || K < 1 || !(p > 0.0) || !(p <= 1.0) || (prec != SV_C128 && prec != SV_C64))
    return SV_E_ARG;
  if (alloc && (!alloc->alloc || !alloc->free)) return SV_E_ARG;
  {  // kernel attributes of the current device (once per device)
    cudaError_t e = sort_prepare();
    if (e == cudaSuccess) e = regroup_prepare();
    if (e == cudaSuccess) e = slots_prepare();
    if (e == cudaSuccess) e = local_prepare();
    if (e == cudaSuccess) e = select_prepare();
    if (e != cudaSuccess) {
      cudaGetLastError();
      return SV_E_CUDA;
    }
  }
  sv_state* s = new sv_state();
  s->n = n;
  s->K = K;
  s->p = p;
  s->prec = prec;
  s->st = (cudaStream_t)cuda_stream;
  s->amp_bytes = prec == SV_C128 ? 16 : 8;
  if (alloc) {
    s->alloc = *alloc;
    s->custom_alloc = true;
  }
  sv_status rc = SV_OK;
  s->hist = (uint32_t*)dev_alloc(s, sizeof(uint32_t) * MAX_PASSES * RADIX);
  s->tile_counter = (uint64_t*)dev_alloc(s, 256);
  s->ctl = (Ctl*)dev_alloc(s, sizeof(Ctl));
  s->ss.hist_count = (uint32_t*)dev_alloc(s, sizeof(uint32_t) * SEL_BINS);
  s->ss.hist_mass = (uint64_t*)dev_alloc(s, sizeof(uint64_t) * 2 * SEL_BINS);
  s->ss.buf = (uint64_t*)dev_alloc(s, sizeof(uint64_t) * 2 * FINISH_CAP);
  if (!s->hist || !s->tile_counter || !s->ctl || !s->ss.hist_count || !s->ss.hist_mass || !s->ss.buf)
    rc = SV_E_NOMEM;
  s->tab_dev = (GateTables*)dev_alloc(s, sizeof(GateTables));
  s->peak_part = (uint64_t*)dev_alloc(s, sizeof(uint64_t) * 2 * PEAK_PARTS);
  if (!s->tab_dev || !s->peak_part) rc = SV_E_NOMEM;
  if (rc == SV_OK && (cudaMallocHost(&s->hist_host, sizeof(uint32_t) * MAX_PASSES * RADIX) != cudaSuccess ||
                      cudaMallocHost(&s->ctl_host, sizeof(Ctl)) != cudaSuccess ||
                      cudaMallocHost(&s->tab_host, sizeof(GateTables)) != cudaSuccess))
    rc = SV_E_CUDA;
  if (rc == SV_OK) rc = ensure_state_cap(s, 4096);
  if (rc == SV_OK) rc = ensure_sort_cap(s, 4096);
  if (rc == SV_OK) {
    cudaMemsetAsync(s->ctl, 0, sizeof(Ctl), s->st);
    // the select histogram starts cleared; each level's pick clears it again
    cudaMemsetAsync(s->ss.hist_count, 0, sizeof(uint32_t) * SEL_BINS, s->st);
    cudaMemsetAsync(s->ss.hist_mass, 0, sizeof(uint64_t) * 2 * SEL_BINS, s->st);
    const uint64_t* nat_dev = &s->tab_dev->nat[0][0];
    cudaMemcpyAsync(&s->ctl->nat, &nat_dev, sizeof(nat_dev), cudaMemcpyHostToDevice, s->st);
    const uint64_t zero_key = 0;
    const double one[2] = {1.0, 0.0};
    const float onef[2] = {1.0f, 0.0f};
    const uint64_t one_bits = 0x3ff0000000000000ull;  // prob of 1+0i
    cudaMemcpyAsync(s->keys[0], &zero_key, 8, cudaMemcpyHostToDevice, s->st);
    cudaMemcpyAsync(s->amps[0], prec == SV_C128 ? (const void*)one : (const void*)onef, s->amp_bytes,
                    cudaMemcpyHostToDevice, s->st);
    cudaMemcpyAsync(s->probs[0], &one_bits, 8, cudaMemcpyHostToDevice, s->st);
    for (int b = 0; b < 64; ++b) s->order[b] = b;
    rc = upload_nat(s);
    if (rc == SV_OK) rc = cuda_check(s, cudaStreamSynchronize(s->st), "sv_create");
    s->N = 1;
    s->cur = 0;
  }
  if (rc != SV_OK) {
    sv_destroy(s);
    return rc;
  }
  *out = s;
  return SV_OK;
}

sv_status sv_create(int n, uint64_t K, double p, sv_state** out) {
  return sv_create_ex(n, K, p, SV_C128, nullptr, nullptr, out);
}

sv_status sv_destroy(sv_state* s) {
  if (!s) return SV_OK;
  if (s->st) cudaStreamSynchronize(s->st);
  else cudaDeviceSynchronize();
  for (int i = 0; i < 2; ++i) {
    dev_free(s, s->keys[i]);
    dev_free(s, s->amps[i]);
    dev_free(s, s->probs[i]);
    dev_free(s, s->sk[i]);
    dev_free(s, s->sidx[i]);
  }
  dev_free(s, s->heads);
  dev_free(s, s->gmask);
  dev_free(s, s->ooff);
  dev_free(s, s->lookback);
  dev_free(s, s->gs_lb);
  dev_free(s, s->hist);
  dev_free(s, s->tile_counter);
  dev_free(s, s->ctl);
  dev_free(s, s->ss.hist_count);
  dev_free(s, s->ss.hist_mass);
  dev_free(s, s->ss.buf);
  dev_free(s, s->ss.win_p);
  dev_free(s, s->ss.win_i);
  dev_free(s, s->ss.tile_keep);
  dev_free(s, s->ss.tile_off);
  dev_free(s, s->ss.keep_bits);
  for (int ph = 0; ph < PH_COUNT; ++ph) {
    if (s->ev_beg[ph]) cudaEventDestroy(s->ev_beg[ph]);
    if (s->ev_end[ph]) cudaEventDestroy(s->ev_end[ph]);
  }
  if (s->hist_host) cudaFreeHost(s->hist_host);
  if (s->peak_host) cudaFreeHost(s->peak_host);
  for (uint32_t i = 0; i < sv_state::PEAK_RING; ++i)
    if (s->peak_ev[i]) cudaEventDestroy(s->peak_ev[i]);
  if (s->ctl_host) cudaFreeHost(s->ctl_host);
  if (s->tab_host) cudaFreeHost(s->tab_host);
  dev_free(s, s->tab_dev);
  dev_free(s, s->peak_part);
  delete s;
  return SV_OK;
}

// Entries (ur[r], ui[r]) that are +-1 or +-i, given which components are
// nonzero (rnz / inz bit r): their products are taken without the FP64 pipe
// (unit), neg when the nonzero component is -1.
static void unit_entries(const double* ur, const double* ui, uint32_t rnz, uint32_t inz, int d, uint32_t* unit,
                         uint32_t* uneg) {
  *unit = *uneg = 0;
  for (int r = 0; r < d; ++r) {
    const bool rz = (rnz >> r) & 1u, iz = (inz >> r) & 1u;
    const double v = rz ? ur[r] : ui[r];
    if (rz != iz && (v == 1.0 || v == -1.0)) {
      *unit |= 1u << r;
      if (v < 0) *uneg |= 1u << r;
    }
  }
}

sv_status sv_apply_gate(sv_state* s, int m, const int* qubits, const double* U) {
  SV_GUARD(s);
  if (m < 1 || m > 4 || !qubits || !U) return fail(s, SV_E_ARG, "sv_apply_gate: bad m or null pointer");
  GateParams gp;
  std::memset(&gp, 0, sizeof(gp));
  gp.m = m;
  gp.rmap = RMAP_IDENTITY;
  gp.n_mask = s->n == 64 ? ~0ull : ((1ull << s->n) - 1);
  for (int t = 0; t < m; ++t) {
    if (qubits[t] < 0 || qubits[t] >= s->n) return fail(s, SV_E_ARG, "sv_apply_gate: qubit out of range");
    if (gp.qmask & (1ull << qubits[t])) return fail(s, SV_E_ARG, "sv_apply_gate: repeated qubit");
    gp.qmask |= 1ull << qubits[t];
    gp.q[t] = qubits[t];
    gp.qs[t] = qubits[t];
  }
  for (int a = 0; a < m; ++a)  // ascending copy
    for (int b = a + 1; b < m; ++b)
      if (gp.qs[b] < gp.qs[a]) {
        int t = gp.qs[a];
        gp.qs[a] = gp.qs[b];
        gp.qs[b] = t;
      }
  if (!is_unitary(m, U)) return fail(s, SV_E_NOT_UNITARY, "sv_apply_gate: U is not unitary within 1e-10");
  const int d = 1 << m;
  for (int ro = 0; ro < d; ++ro)
    for (int r = 0; r < d; ++r) {
      double ur = U[2 * (ro * d + r)], ui = U[2 * (ro * d + r) + 1];
      s->tab_host->U[2 * (ro * d + r)] = ur;  // uploaded with the permutation
      s->tab_host->U[2 * (ro * d + r) + 1] = ui;
      // complex64: the zero pattern is that of the float-rounded entries
      bool rz = s->prec == SV_C128 ? ur != 0.0 : (float)ur != 0.0f;
      bool iz = s->prec == SV_C128 ? ui != 0.0 : (float)ui != 0.0f;
      if (rz) gp.re_nz[ro] |= 1u << r;
      if (iz) gp.im_nz[ro] |= 1u << r;
    }
  // One nonzero per row and column (a permutation with phases): every term
  // has one output, r -> pi(r), kept in nibble r of pi.
  bool mono = true;
  uint64_t pi = 0;
  uint32_t cols_seen = 0;
  for (int ro = 0; ro < d && mono; ++ro) {
    const uint32_t row = gp.re_nz[ro] | gp.im_nz[ro];
    const int r = row ? __builtin_ctz(row) : 0;
    if (__builtin_popcount(row) != 1 || ((cols_seen >> r) & 1u)) {
      mono = false;
    } else {
      cols_seen |= 1u << r;
      pi |= (uint64_t)ro << (4 * r);
    }
  }
  const uint64_t N = s->N;
  s->peak_ready = false;
  s->total_ready = false;
  s->stats.n_in = N;
  s->stats.sort_passes = 0;
  if (N == 0) {
    s->stats.n_pre = 0;
    return SV_OK;
  }
  if (N > MAX_TERMS || (N << m) > MAX_TERMS * 16ull)
    return fail(s, SV_E_ARG, "sv_apply_gate: state too large for 32-bit term indices");
  sv_status rc = ensure_state_cap(s, N << m);
  if (rc == SV_OK) rc = ensure_sort_cap(s, N);
  if (rc != SV_OK) return rc;
  const uint64_t gs_words = group_scan_lookback_words(N);  // the group scan's two look-backs
  rc = ensure_gs_lb(s, gs_words);
  if (rc != SV_OK) return rc;
  const int alt = 1 - s->cur;
  for (int b = 0; b < s->n; ++b) s->order_next[b] = s->order[b];
  // A diagonal U maps every term to itself (Eq. 3 with no off-diagonal
  // entries): no grouping, the amplitudes are updated in place and the
  // state keeps its order (default variant; the others regroup as always).
  bool diag = s->variant == 0;
  for (int ro = 0; ro < d && diag; ++ro)
    if ((gp.re_nz[ro] | gp.im_nz[ro]) & ~(1u << ro)) diag = false;
  if (diag) {
    DiagParams dp;
    std::memset(&dp, 0, sizeof(dp));
    dp.m = m;
    for (int t = 0; t < m; ++t) dp.qpos[t] = s->order[gp.q[t]];
    for (int r = 0; r < d; ++r) {
      dp.ur[r] = U[2 * (r * d + r)];
      dp.ui[r] = U[2 * (r * d + r) + 1];
      dp.rnz |= gp.re_nz[r] & (1u << r);
      dp.inz |= gp.im_nz[r] & (1u << r);
    }
    unit_entries(dp.ur, dp.ui, dp.rnz, dp.inz, d, &dp.unit, &dp.uneg);
    ++s->global_gates;
    ++s->stats.diag_gates;
    // clears the gate's counters (zero count, total mass); no table to store
    launch_store_tables(*s->tab_host, s->tab_dev, 0, GateReset{s->ctl, s->hist, nullptr, 0}, s->st);
    ph_begin(s, PH_APPLY);
    launch_diag_apply(s->prec, s->keys[s->cur], s->amps[s->cur], s->probs[s->cur], N, dp, s->ctl, s->st);
    ph_end(s, PH_APPLY);
    launched(s, PH_APPLY, 2);
    rc = sync_ctl(s, "sv_apply_gate");
    if (rc != SV_OK) return rc;
    if (s->ctl_host->count[3] != 0) {  // exact zeros: drop them in order
      rc = ensure_lookback(s, N / 2048 + 16);
      if (rc != SV_OK) return rc;
      ph_begin(s, PH_APPLY);
      launch_drop_zero_terms(s->prec, s->keys[s->cur], s->amps[s->cur], s->probs[s->cur], N, s->keys[alt],
                             s->amps[alt], s->probs[alt], s->lookback, s->ctl, s->st);
      ph_end(s, PH_APPLY);
      launched(s, PH_APPLY, 1);
      rc = sync_ctl(s, "sv_apply_gate");
      if (rc != SV_OK) return rc;
      s->cur = alt;
      s->N = s->ctl_host->count[2];
    }
    s->total_ready = true;
    s->probs_valid = true;  // the diagonal kernel rewrote every probability
    ++s->gate_index;
    s->stats.n_pre = s->N;
    s->stats.local_gates = s->local_gates;
    s->stats.global_gates = s->global_gates;
    s->stats.local_fallbacks = s->local_fallbacks;
    return SV_OK;
  }
  // The bucket-local kernel sorts and applies inside shared memory; it is used
  // for states that fit one of its batches (measured: beyond that the sorted
  // path was as fast or faster on this GPU, without bucket bookkeeping).
  const bool local = s->variant != 1 && N <= LOCAL_BUCKET_MAX;
  static const bool debug = getenv("SV_DEBUG") != nullptr;
  if (debug)
    fprintf(stderr, "[sv] gate %lld N=%llu q=(%d,%d) -> %s\n", (long long)s->gate_index, (unsigned long long)N,
            gp.q[0], m > 1 ? gp.q[1] : -1, local ? "local" : "global");
  bool done = false;
  if (local) {
    rc = upload_perm(s, gp);
    if (rc != SV_OK) return rc;
    ph_begin(s, PH_LOCAL);
    launch_local_gate(s->prec, s->keys[s->cur], s->amps[s->cur], N, gp, s->keys[alt], s->amps[alt],
                      s->probs[alt], s->ctl, s->st);
    ph_end(s, PH_LOCAL);
    launched(s, PH_LOCAL, 1);
    rc = sync_ctl(s, "sv_apply_gate");
    if (rc != SV_OK) return rc;
    if (s->ctl_host->err & ERR_BUCKET) {  // a bucket outgrew the batch limit: redo globally
      ++s->local_fallbacks;
      rc = cuda_check(s, cudaMemsetAsync(&s->ctl->err, 0, sizeof(uint32_t), s->st), "sv_apply_gate");
      if (rc != SV_OK) return rc;
    } else {
      ++s->local_gates;
      done = true;
      const uint64_t npre = s->ctl_host->count[1];
      if (s->ctl_host->count[3] != 0) {  // exact cancellations: drop the zero terms
        rc = ensure_lookback(s, npre / 2048 + 16);
        if (rc != SV_OK) return rc;
        ph_begin(s, PH_APPLY);
        launch_drop_zero_terms(s->prec, s->keys[alt], s->amps[alt], s->probs[alt], npre, s->keys[s->cur],
                               s->amps[s->cur], s->probs[s->cur], s->lookback, s->ctl, s->st);
        ph_end(s, PH_APPLY);
        launched(s, PH_APPLY, 1);
        rc = sync_ctl(s, "sv_apply_gate");
        if (rc != SV_OK) return rc;
        s->N = s->ctl_host->count[2];
      } else {
        s->cur = alt;
        s->N = npre;
      }
    }
  }
  if (!done && s->variant == 1) {
    // expand-first: one record per (term, output) pair, sorted by (output, source r), then
    // one fused multiply-add chain per output
    ++s->global_gates;
    const uint64_t nrec = N << m;
    rc = ensure_sort_cap(s, nrec);
    const uint64_t red_tiles = nrec / 1024 + 2;
    if (rc == SV_OK) rc = ensure_lookback(s, red_tiles + 16);
    if (rc != SV_OK) return rc;
    rc = upload_perm(s, gp);
    if (rc != SV_OK) return rc;
    const int nbits = s->n + m;
    const int passes = (nbits + RADIX_BITS - 1) / RADIX_BITS;
    ph_begin(s, PH_KEYS);
    launch_expand_records(s->keys[s->cur], N, gp, s->sk[0], s->sidx[0], s->hist, passes, s->st);
    ph_end(s, PH_KEYS);
    launched(s, PH_KEYS, 1);
    int w = 0, run = 0;
    rc = sort_pairs(s, nrec, nbits, true, &w, &run);
    if (rc != SV_OK) return rc;
    s->stats.sort_passes = (uint32_t)run;
    ph_begin(s, PH_HEADS);
    launch_group_heads(s->sk[w], nrec, m, s->heads, s->lookback, s->ctl, s->st);
    ph_end(s, PH_HEADS);
    ph_begin(s, PH_APPLY);
    launch_segment_reduce(s->prec, s->sk[w], s->sidx[w], nrec, s->heads, s->amps[s->cur], gp, s->keys[alt],
                          s->amps[alt], s->probs[alt], s->lookback, s->ctl, red_tiles, s->st);
    ph_end(s, PH_APPLY);
    launched(s, PH_HEADS, 1);
    launched(s, PH_APPLY, 1);
    rc = sync_ctl(s, "sv_apply_gate");
    if (rc != SV_OK) return rc;
    s->cur = alt;
    s->N = s->ctl_host->count[1];
    done = true;
  }
  if (!done) {
    ++s->global_gates;
    rc = upload_perm(s, gp, GateReset{s->ctl, s->hist, s->gs_lb, (uint32_t)gs_words});
    if (rc != SV_OK) return rc;
    const int passes = (s->n + RADIX_BITS - 1) / RADIX_BITS;
    // pack the term index below the sort key when both fit in 64 bits
    int vbits = 1;
    while (vbits < 63 && (N - 1) >> vbits) ++vbits;
    gp.vbits = s->n + vbits <= 64 ? vbits : 0;
    int w = 0, run = 0;
    // monomial gates on the default variant: the partition digit is the output
    // index, so the merged keys come out in the output order
    const bool mono_path = mono && s->variant == 0;
    if (mono_path) gp.rmap = pi;
    if (s->variant == 0) {
      // the state is sorted by the previous gate's key: partition by the gate
      // bits and merge
      cudaError_t e;
      int nl = 0;
      ph_begin(s, PH_SORT);
      w = regroup_terms(s->keys[s->cur], N, gp, s->sk, s->sidx, sort_scratch(s), s->st, &nl, &e);
      ph_end(s, PH_SORT);
      launched(s, PH_SORT, (uint64_t)nl);
      rc = cuda_check(s, e, "regroup");
      if (rc != SV_OK) return rc;
      run = 1 + m;
    } else {
      ph_begin(s, PH_KEYS);
      launch_gate_keys(s->keys[s->cur], N, gp, s->sk[0], s->sidx[0], s->hist, passes, s->st);
      ph_end(s, PH_KEYS);
      launched(s, PH_KEYS, 1);
      rc = gp.vbits ? sort_keys(s, N, gp.vbits, s->n, &w, &run) : sort_pairs(s, N, s->n, true, &w, &run);
      if (rc != SV_OK) return rc;
    }
    s->stats.sort_passes = (uint32_t)run;
    uint64_t npre = N;
    if (mono_path) {
      ++s->stats.mono_gates;
      // the regrouping sorted the terms by output key: one output per term
      MonoParams mp;
      std::memset(&mp, 0, sizeof(mp));
      mp.m = m;
      mp.vbits = gp.vbits;
      for (int r = 0; r < d; ++r) {
        const int ro = (int)((pi >> (4 * r)) & 15u);
        mp.ur[ro] = U[2 * (ro * d + r)];
        mp.ui[ro] = U[2 * (ro * d + r) + 1];
        mp.rnz |= ((gp.re_nz[ro] >> r) & 1u) << ro;
        mp.inz |= ((gp.im_nz[ro] >> r) & 1u) << ro;
      }
      unit_entries(mp.ur, mp.ui, mp.rnz, mp.inz, d, &mp.unit, &mp.uneg);
      ph_begin(s, PH_APPLY);
      launch_mono_apply(s->prec, s->sk[w], s->sidx[w], N, s->amps[s->cur], mp, s->keys[alt], s->amps[alt],
                        s->probs[alt], s->ctl, s->st);
      s->total_ready = true;  // zeros dropped below add no mass
      ph_end(s, PH_APPLY);
      launched(s, PH_APPLY, 1);
      rc = sync_ctl(s, "sv_apply_gate");
      if (rc != SV_OK) return rc;
    } else {
      ph_begin(s, PH_HEADS);
      launch_group_scan(s->sk[w], N, gp, s->heads, s->gmask, s->ooff, s->gs_lb, s->ctl, s->st);
      ph_end(s, PH_HEADS);
      ph_begin(s, PH_APPLY);
      launch_gate_apply_slots(s->prec, s->sk[w], s->sidx[w], N, s->heads, s->gmask, s->ooff, s->amps[s->cur], gp,
                              s->keys[alt], s->amps[alt], s->probs[alt], s->ctl, s->st);
      s->total_ready = s->prec == SV_C128;  // zeros dropped below add no mass
      ph_end(s, PH_APPLY);
      launched(s, PH_HEADS, 1);
      launched(s, PH_APPLY, 1);
      rc = sync_ctl(s, "sv_apply_gate");
      if (rc != SV_OK) return rc;
      npre = s->ctl_host->count[1];
    }
    if (s->ctl_host->count[3] != 0) {  // exact cancellations: drop the zero terms in order
      rc = ensure_lookback(s, npre / 2048 + 16);
      if (rc != SV_OK) return rc;
      ph_begin(s, PH_APPLY);
      launch_drop_zero_terms(s->prec, s->keys[alt], s->amps[alt], s->probs[alt], npre, s->keys[s->cur],
                             s->amps[s->cur], s->probs[s->cur], s->lookback, s->ctl, s->st);
      ph_end(s, PH_APPLY);
      launched(s, PH_APPLY, 1);
      rc = sync_ctl(s, "sv_apply_gate");
      if (rc != SV_OK) return rc;
      s->N = s->ctl_host->count[2];
    } else {
      s->cur = alt;
      s->N = npre;
    }
  }
  ++s->gate_index;
  s->probs_valid = true;  // every gate path writes all its outputs' probabilities
  for (int b = 0; b < s->n; ++b) s->order[b] = s->order_next[b];
  s->stats.n_pre = s->N;
  s->stats.local_gates = s->local_gates;
  s->stats.global_gates = s->global_gates;
  s->stats.local_fallbacks = s->local_fallbacks;
  return SV_OK;
}

}  // extern "C"

namespace {

// Window buffer for the truncation select: room for N/6 + 65536 terms.
sv_status ensure_window_cap(sv_state* s, uint64_t N) {
  uint64_t need = N / 6 + 65536;
  if (need > s->ss.win_cap) {
    uint64_t cap = need + need / 2;
    dev_free(s, s->ss.win_p);
    dev_free(s, s->ss.win_i);
    s->ss.win_p = (uint64_t*)dev_alloc(s, cap * 8);
    s->ss.win_i = (uint32_t*)dev_alloc(s, cap * 4);
    if (!s->ss.win_p || !s->ss.win_i) {
      s->ss.win_cap = 0;
      return fail(s, SV_E_NOMEM, "select window allocation failed");
    }
    s->ss.win_cap = cap;
  }
  uint64_t tiles = window_tiles(N) + 1;
  if (tiles > s->ss.tiles_cap) {
    uint64_t cap = tiles + tiles / 2 + 64;
    dev_free(s, s->ss.tile_keep);
    dev_free(s, s->ss.tile_off);
    dev_free(s, s->ss.keep_bits);
    s->ss.tile_keep = (uint32_t*)dev_alloc(s, cap * 4);
    s->ss.tile_off = (uint64_t*)dev_alloc(s, cap * 8);
    s->ss.keep_bits = (uint32_t*)dev_alloc(s, cap * (WINDOW_TILE / 32) * 4);
    if (!s->ss.tile_keep || !s->ss.tile_off || !s->ss.keep_bits) {
      s->ss.tiles_cap = 0;
      return fail(s, SV_E_NOMEM, "select tile table allocation failed");
    }
    s->ss.tiles_cap = cap;
  }
  return SV_OK;
}

// Exact cut by count (mode 1, rank count_target) or by mass (mode 0, p of
// the total): sample window + one streaming pass, then radix-select levels on
// the window (or on all terms when the window misses).  The result is left
// in s->ctl_host.
sv_status run_select(sv_state* s, int mode, uint64_t count_target, uint32_t* levels) {
  const uint64_t N = s->N;
  ensure_probs(s);
  sv_status rc = ensure_window_cap(s, N);
  if (rc != SV_OK) return rc;
  ph_begin(s, PH_WINDOW);
  launch_select_window(s->probs[s->cur], s->keys[s->cur], N, s->ctl, s->ss, mode, count_target, s->p, s->total_ready,
                       s->st);
  s->total_ready = true;  // the pass summed the total when it was not known: a second select reuses it
  ph_end(s, PH_WINDOW);
  launched(s, PH_WINDOW, 3);
  // Two levels and the finish are enqueued behind the window without a host
  // wait: the kernels read on the device whether the window was taken, how
  // long the list is and whether the bin is small enough to finish; the host
  // continues level by level only when that did not resolve the cut.
  ph_begin(s, PH_SELECT);
  for (int level = 0; level < 2; ++level) {
    launch_select_hist(s->probs[s->cur], s->keys[s->cur], N, s->ctl, s->ss, s->st);
    launch_select_pick(s->ctl, s->ss, s->p, s->st);
  }
  launch_select_compact(s->probs[s->cur], s->keys[s->cur], N, s->ctl, s->ss, s->st);
  launch_select_finish(s->ctl, s->ss, s->p, s->st);
  ph_end(s, PH_SELECT);
  launched(s, PH_SELECT, 6);
  *levels += 2;
  rc = sync_ctl(s, "truncation select");
  if (rc != SV_OK) return rc;
  s->stats.window_terms = s->ctl_host->win_n;
  s->stats.window_hits += s->ctl_host->use_window ? 1 : 0;
  if (s->ctl_host->sel_done) return SV_OK;
  bool small = s->ctl_host->sel_bin_count <= (uint64_t)FINISH_CAP;
  for (int level = 0; level < 16; ++level) {
    if (!small) {
      ph_begin(s, PH_SELECT);
      launch_select_hist(s->probs[s->cur], s->keys[s->cur], N, s->ctl, s->ss, s->st);
      launch_select_pick(s->ctl, s->ss, s->p, s->st);
      ph_end(s, PH_SELECT);
      launched(s, PH_SELECT, 2);
      ++*levels;
      rc = sync_ctl(s, "truncation select");
      if (rc != SV_OK) return rc;
      if (s->ctl_host->sel_done) return SV_OK;
      small = s->ctl_host->sel_bin_count <= (uint64_t)FINISH_CAP;
    }
    if (small) {
      ph_begin(s, PH_SELECT);
      launch_select_compact(s->probs[s->cur], s->keys[s->cur], N, s->ctl, s->ss, s->st);
      launch_select_finish(s->ctl, s->ss, s->p, s->st);
      ph_end(s, PH_SELECT);
      launched(s, PH_SELECT, 2);
      rc = sync_ctl(s, "truncation select");
      if (rc != SV_OK) return rc;
      if (!s->ctl_host->sel_done) {
        s->broken = true;
        return fail(s, SV_E_STATE, "truncation select did not resolve");
      }
      return SV_OK;
    }
  }
  s->broken = true;
  return fail(s, SV_E_STATE, "truncation select did not resolve");
}

}  // namespace

extern "C" {

sv_status sv_truncate(sv_state* s, uint64_t* kept, double* retained_fraction) {
  SV_GUARD(s);
  const uint64_t N = s->N;
  s->stats.select_levels = 0;
  s->stats.window_hits = 0;
  s->stats.window_terms = 0;
  s->stats.selects = 0;
  s->stats.n_kept = N;
  s->stats.total_mass = s->stats.kept_mass = 0.0;
  const bool need_p = s->p < 1.0, need_k = N > s->K;
  double f = 1.0;
  if (N > 0 && (need_p || need_k)) {
    uint64_t c = N;
    bool have_cut = false;
    sv_status rc;
    // c = min(c_p, K).  With more than K terms the top-k cut is found first:
    // its kept mass S_K decides whether the p-mass cut can lie before it
    // (c_p <= K exactly when S_K >= T, the prefix masses being monotone), so
    // the p-mass select runs only then.
    bool run_p = need_p;
    if (need_k) {
      rc = run_select(s, 1, s->K, &s->stats.select_levels);
      if (rc != SV_OK) return rc;
      ++s->stats.selects;
      if (s->ctl_host->sel_done != 1) {
        s->broken = true;
        return fail(s, SV_E_STATE, "top-k select found no cut");
      }
      c = s->ctl_host->cut_count;
      have_cut = true;
      if (need_p) {
        const double SNd = u128_to_double(s->ctl_host->total_mass_hi, s->ctl_host->total_mass_lo);
        const unsigned __int128 T = fx_from_double(s->p * SNd);
        const unsigned __int128 SK =
            ((unsigned __int128)s->ctl_host->cut_mass_hi << 64) | s->ctl_host->cut_mass_lo;
        run_p = SK >= T;
      }
    }
    if (run_p) {
      rc = run_select(s, 0, 0, &s->stats.select_levels);
      if (rc != SV_OK) return rc;
      ++s->stats.selects;
      if (s->ctl_host->sel_done == 1) {
        c = s->ctl_host->cut_count;
        have_cut = true;
      } else if (need_k) {
        s->broken = true;
        return fail(s, SV_E_STATE, "p-mass select found no cut below the top-k cut");
      }
    }
    double SN = u128_to_double(s->ctl_host->total_mass_hi, s->ctl_host->total_mass_lo);
    s->stats.total_mass = SN;
    s->stats.kept_mass = SN;
    if (have_cut && c < N) {
      const int alt = 1 - s->cur;
      rc = ensure_lookback(s, (N + 1023) / 1024 + 16);
      if (rc != SV_OK) return rc;
      ph_begin(s, PH_COMPACT);
      if (s->ctl_host->use_window) {
        launch_truncate_windowed(s->prec, s->keys[s->cur], s->amps[s->cur], s->probs[s->cur], N,
                                 s->keys[alt], s->amps[alt], s->ss, s->ctl, s->st, s->peak_part, &s->peak_blocks);
        launched(s, PH_COMPACT, 3);
      } else {
        launch_set_scale(s->ctl, s->st);
        launch_truncate_compact(s->prec, s->keys[s->cur], s->amps[s->cur], s->probs[s->cur], N,
                                s->keys[alt], s->amps[alt], s->lookback, s->ctl, s->st, s->peak_part,
                                &s->peak_blocks);
        launched(s, PH_COMPACT, 2);
      }
      ph_end(s, PH_COMPACT);
      // no wait here: the next wait on the stream checks the count written
      rc = cuda_check(s, cudaMemcpyAsync(&s->ctl->kept_check, &s->ctl->count[2], sizeof(uint64_t),
                                         cudaMemcpyDeviceToDevice, s->st),
                      "sv_truncate");
      if (rc != SV_OK) return rc;
      s->kept_pending = true;
      s->kept_expected = c;
      s->peak_ready = s->peak_blocks > 0;
      s->total_ready = false;
      double Sc = u128_to_double(s->ctl_host->cut_mass_hi, s->ctl_host->cut_mass_lo);
      f = Sc / SN;
      s->F = s->F * f;
      s->cur = alt;
      s->probs_valid = false;
      s->N = c;
      s->stats.kept_mass = Sc;
    }
  }
  s->stats.n_kept = s->N;
  if (kept) *kept = s->N;
  if (retained_fraction) *retained_fraction = f;
  return SV_OK;
}

sv_status sv_select_histogram(sv_state* s, uint64_t prefix_hi, uint64_t prefix_lo, int bits, uint32_t* counts,
                              uint64_t* masses) {
  SV_GUARD(s);
  if (bits < 0 || bits > 127 || !counts || !masses) return fail(s, SV_E_ARG, "sv_select_histogram: bad arguments");
  std::memset(counts, 0, sizeof(uint32_t) * SEL_BINS);
  std::memset(masses, 0, sizeof(uint64_t) * 2 * SEL_BINS);
  if (s->N == 0) return SV_OK;
  // the histogram arrays arrive cleared (the pick of every select level
  // clears them) and are cleared again after the copy
  ensure_probs(s);
  launch_set_select(s->ctl, prefix_hi, prefix_lo, (uint32_t)bits, s->st);
  launch_select_hist(s->probs[s->cur], s->keys[s->cur], s->N, s->ctl, s->ss, s->st);
  launched(s, PH_SELECT, 2);
  cudaError_t e = cudaMemcpyAsync(counts, s->ss.hist_count, sizeof(uint32_t) * SEL_BINS, cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(masses, s->ss.hist_mass, sizeof(uint64_t) * 2 * SEL_BINS, cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->ss.hist_count, 0, sizeof(uint32_t) * SEL_BINS, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->ss.hist_mass, 0, sizeof(uint64_t) * 2 * SEL_BINS, s->st);
  g_d2h += sizeof(uint32_t) * SEL_BINS + sizeof(uint64_t) * 2 * SEL_BINS;
  sv_status rc = cuda_check(s, e, "sv_select_histogram");
  if (rc != SV_OK) return rc;
  return sync_ctl(s, "sv_select_histogram");
}

sv_status sv_cut(sv_state* s, uint64_t z_hi, uint64_t z_lo, uint64_t sc_hi, uint64_t sc_lo, uint64_t sn_hi,
                 uint64_t sn_lo, uint64_t* kept) {
  SV_GUARD(s);
  if ((sc_hi | sc_lo) == 0 || (sn_hi | sn_lo) == 0) return fail(s, SV_E_ARG, "sv_cut: zero mass");
  const double Sc = u128_to_double(sc_hi, sc_lo), SN = u128_to_double(sn_hi, sn_lo);
  s->peak_ready = false;
  s->total_ready = false;
  const uint64_t N = s->N;
  if (N > 0) {
    const int alt = 1 - s->cur;
    sv_status rc = ensure_lookback(s, (N + 1023) / 1024 + 16);
    if (rc != SV_OK) return rc;
    ph_begin(s, PH_COMPACT);
    ensure_probs(s);
    launch_set_cut(s->ctl, ~z_hi, z_lo, sc_hi, sc_lo, s->st);
    launch_set_scale(s->ctl, s->st);
    launch_truncate_compact(s->prec, s->keys[s->cur], s->amps[s->cur], s->probs[s->cur], N, s->keys[alt],
                            s->amps[alt], s->lookback, s->ctl, s->st, s->peak_part, &s->peak_blocks);
    ph_end(s, PH_COMPACT);
    launched(s, PH_COMPACT, 3);
    rc = sync_ctl(s, "sv_cut");
    if (rc != SV_OK) return rc;
    s->cur = alt;
    s->N = s->ctl_host->count[2];
    s->peak_ready = s->peak_blocks > 0 && s->N > 0;
    s->probs_valid = false;
  }
  s->F = s->F * (Sc / SN);
  s->stats.n_kept = s->N;
  if (kept) *kept = s->N;
  return SV_OK;
}

namespace {
void enqueue_peak(sv_state* s) {
  ph_begin(s, PH_PEAK);
  if (s->peak_ready) {  // the last truncation's compaction left per-block partials
    launch_peak_partials(s->peak_part, s->peak_blocks, s->ctl, s->st);
    launched(s, PH_PEAK, 1);
  } else {
    ensure_probs(s);
    launch_peak(s->probs[s->cur], s->keys[s->cur], s->N, s->ctl, s->st);
    launched(s, PH_PEAK, 2);
  }
  ph_end(s, PH_PEAK);
}
}  // namespace

sv_status sv_peak(sv_state* s, uint64_t* key, double* prob) {
  SV_GUARD(s);
  if (!key || !prob) return fail(s, SV_E_ARG, "sv_peak: null output");
  if (s->N == 0) return fail(s, SV_E_STATE, "sv_peak: empty state");
  enqueue_peak(s);
  sv_status rc = sync_ctl(s, "sv_peak");
  if (rc != SV_OK) return rc;
  *key = s->ctl_host->peak_z_lo;
  uint64_t b = s->ctl_host->peak_z_hi;
  std::memcpy(prob, &b, 8);
  return SV_OK;
}

sv_status sv_peak_async(sv_state* s, uint64_t* ticket) {
  SV_GUARD(s);
  if (!ticket) return fail(s, SV_E_ARG, "sv_peak_async: null ticket");
  if (s->N == 0) return fail(s, SV_E_STATE, "sv_peak_async: empty state");
  if (!s->peak_host) {
    if (cudaMallocHost(&s->peak_host, sizeof(uint64_t) * 2 * sv_state::PEAK_RING) != cudaSuccess) {
      s->peak_host = nullptr;
      return fail(s, SV_E_NOMEM, "sv_peak_async: pinned result ring");
    }
    for (uint32_t i = 0; i < sv_state::PEAK_RING; ++i) {
      sv_status rc = cuda_check(s, cudaEventCreateWithFlags(&s->peak_ev[i], cudaEventDisableTiming),
                                "sv_peak_async");
      if (rc != SV_OK) return rc;
    }
  }
  enqueue_peak(s);
  const uint64_t t = s->peak_issued++;
  const uint32_t slot = (uint32_t)(t % sv_state::PEAK_RING);
  sv_status rc = cuda_check(s, cudaMemcpyAsync(s->peak_host + 2 * slot, &s->ctl->peak_z_hi, 2 * sizeof(uint64_t),
                                               cudaMemcpyDeviceToHost, s->st),
                            "sv_peak_async");
  if (rc == SV_OK) rc = cuda_check(s, cudaEventRecord(s->peak_ev[slot], s->st), "sv_peak_async");
  if (rc != SV_OK) return rc;
  *ticket = t;
  return SV_OK;
}

sv_status sv_peak_wait(sv_state* s, uint64_t ticket, uint64_t* key, double* prob) {
  SV_GUARD(s);
  if (!key || !prob) return fail(s, SV_E_ARG, "sv_peak_wait: null output");
  if (ticket >= s->peak_issued || s->peak_issued - ticket > sv_state::PEAK_RING)
    return fail(s, SV_E_ARG, "sv_peak_wait: unknown ticket or result already overwritten");
  const uint32_t slot = (uint32_t)(ticket % sv_state::PEAK_RING);
  // only this result's copy is waited for (device error flags are checked
  // at the next wait of the other calls)
  sv_status rc = cuda_check(s, cudaEventSynchronize(s->peak_ev[slot]), "sv_peak_wait");
  if (rc != SV_OK) return rc;
  *key = s->peak_host[2 * slot + 1];
  std::memcpy(prob, &s->peak_host[2 * slot], 8);
  return SV_OK;
}

sv_status sv_num_terms(sv_state* s, uint64_t* N) {
  SV_GUARD(s);
  if (!N) return SV_E_ARG;
  *N = s->N;
  return SV_OK;
}

sv_status sv_retained_mass(sv_state* s, double* F) {
  SV_GUARD(s);
  if (!F) return SV_E_ARG;
  *F = s->F;
  return SV_OK;
}

static sv_status dump(sv_state* s, uint64_t* keys, double* amps, double* probs, uint64_t cap,
                      uint64_t* count) {
  SV_GUARD(s);
  if (!count) return fail(s, SV_E_ARG, "null count");
  const uint64_t N = s->N;
  *count = N;
  const uint64_t w = cap < N ? cap : N;
  if (w == 0) return SV_OK;
  int which = 0;
  sv_status rc = canonical_perm(s, &which);
  if (rc != SV_OK) return rc;
  uint64_t* dk = nullptr;
  double* da = nullptr;
  uint64_t* dp = nullptr;
  const int alt = 1 - s->cur;
  if (keys) dk = s->keys[alt];
  if (probs) dp = s->probs[alt];
  void* tmp = nullptr;
  if (amps) {
    tmp = dev_alloc(s, w * 16);
    if (!tmp) return fail(s, SV_E_NOMEM, "export buffer allocation failed");
    da = (double*)tmp;
  }
  launch_gather_terms(s->prec, s->sidx[which], w, s->keys[s->cur], s->amps[s->cur], s->probs[s->cur],
                      dk, da, dp, s->ctl, s->st);
  launched(s, PH_OTHER, 1);
  g_d2h += w * ((dk ? 8 : 0) + (dp ? 8 : 0) + (da ? 16 : 0));
  if (dk) cudaMemcpyAsync(keys, dk, w * 8, cudaMemcpyDeviceToHost, s->st);
  if (dp) cudaMemcpyAsync(probs, dp, w * 8, cudaMemcpyDeviceToHost, s->st);
  if (da) cudaMemcpyAsync(amps, da, w * 16, cudaMemcpyDeviceToHost, s->st);
  rc = cuda_check(s, cudaStreamSynchronize(s->st), "export");
  if (tmp) dev_free(s, tmp);
  return rc;
}

sv_status sv_probs(sv_state* s, uint64_t* keys, double* probs, uint64_t cap, uint64_t* count) {
  return dump(s, keys, nullptr, probs, cap, count);
}

sv_status sv_export(sv_state* s, uint64_t* keys, double* amps, uint64_t cap, uint64_t* count) {
  return dump(s, keys, amps, nullptr, cap, count);
}

sv_status sv_load(sv_state* s, const uint64_t* keys, const double* amps, uint64_t N) {
  SV_GUARD(s);
  s->peak_ready = false;
  s->total_ready = false;
  if (N > 0 && (!keys || !amps)) return fail(s, SV_E_ARG, "sv_load: null input");
  if (N > MAX_TERMS) return fail(s, SV_E_ARG, "sv_load: too many terms");
  if (s->n < 64)
    for (uint64_t i = 0; i < N; ++i)
      if (keys[i] >> s->n) return fail(s, SV_E_ARG, "sv_load: key outside n bits");
  sv_status rc = ensure_state_cap(s, N);
  if (rc == SV_OK) rc = ensure_sort_cap(s, N);
  if (rc == SV_OK) rc = ensure_lookback(s, (N + 1023) / 1024 + 16);
  if (rc != SV_OK) return rc;
  if (N == 0) {
    s->N = 0;
    s->probs_valid = true;
    return SV_OK;
  }
  double* tmp = (double*)dev_alloc(s, N * 16);
  if (!tmp) return fail(s, SV_E_NOMEM, "sv_load: staging allocation failed");
  g_h2d += N * 24;
  cudaMemcpyAsync(s->sk[0], keys, N * 8, cudaMemcpyHostToDevice, s->st);
  cudaMemcpyAsync(tmp, amps, N * 16, cudaMemcpyHostToDevice, s->st);
  launch_iota(s->sidx[0], N, s->st);
  launched(s, PH_OTHER, 1);
  int w = 0, passes = 0;
  rc = sort_pairs(s, N, s->n, false, &w, &passes);
  if (rc != SV_OK) {
    dev_free(s, tmp);
    return rc;
  }
  const int alt = 1 - s->cur;
  launch_load_compact(s->prec, s->sk[w], s->sidx[w], N, tmp, s->keys[alt], s->amps[alt], s->probs[alt],
                      s->lookback, s->ctl, s->st);
  launched(s, PH_OTHER, 1);
  rc = sync_ctl(s, "sv_load");
  dev_free(s, tmp);
  if (rc != SV_OK) return rc;
  if (s->ctl_host->count[3] != 0) return fail(s, SV_E_ARG, "sv_load: duplicate keys");
  s->cur = alt;
  s->N = s->ctl_host->count[2];
  s->probs_valid = true;  // written by the load's compaction
  for (int b = 0; b < 64; ++b) s->order[b] = b;  // sorted by key, stored as natural keys
  rc = upload_nat(s);
  if (rc != SV_OK) return rc;
  return SV_OK;
}

const char* sv_last_error(const sv_state* s) {
  if (!s) return "null handle";
  return s->err.c_str();
}

sv_status sv_last_stats(const sv_state* s, sv_stats* out) {
  if (!s || !out) return SV_E_ARG;
  *out = s->stats;
  return SV_OK;
}

sv_status sv_reserve(sv_state* s, uint64_t terms) {
  SV_GUARD(s);
  if (terms > MAX_TERMS) return fail(s, SV_E_ARG, "sv_reserve: more terms than 32-bit term indices allow");
  if (terms == 0) return SV_OK;
  const uint64_t cand = terms << 4;  // a 4-qubit gate gives each term at most 16 candidates
  sv_status rc = ensure_state_cap(s, cand);
  if (rc == SV_OK) rc = ensure_sort_cap(s, terms);
  if (rc == SV_OK) rc = ensure_gs_lb(s, group_scan_lookback_words(terms));
  if (rc == SV_OK) rc = ensure_window_cap(s, cand);
  if (rc == SV_OK) rc = ensure_lookback(s, (cand + 1023) / 1024 + 16);
  if (rc == SV_OK) rc = cuda_check(s, cudaStreamSynchronize(s->st), "sv_reserve");
  return rc;
}

sv_status sv_set_apply_variant(sv_state* s, int variant) {
  SV_GUARD(s);
  if (variant < 0 || variant > 2) return fail(s, SV_E_ARG, "sv_set_apply_variant: variant must be 0, 1 or 2");
  s->variant = variant;
  return SV_OK;
}

sv_status sv_set_timing(sv_state* s, int enable) {
  if (!s) return SV_E_ARG;
  if (enable && !s->ev_beg[0]) {
    for (int ph = 0; ph < PH_COUNT; ++ph) {
      if (cudaEventCreate(&s->ev_beg[ph]) != cudaSuccess || cudaEventCreate(&s->ev_end[ph]) != cudaSuccess)
        return fail(s, SV_E_CUDA, "sv_set_timing: event creation failed");
    }
  }
  s->timing = enable != 0;
  for (int ph = 0; ph < PH_COUNT; ++ph) {
    s->ph_ms[ph] = 0.0;
    s->ph_launches[ph] = 0;
    s->ph_pending[ph] = false;
  }
  return SV_OK;
}

sv_status sv_phase_times(const sv_state* s, double* ms, uint64_t* launches) {
  if (!s) return SV_E_ARG;
  if (s->timing) {  // fold in the phases still pending on the stream (the last compaction)
    sv_state* w = const_cast<sv_state*>(s);
    if (cudaStreamSynchronize(w->st) == cudaSuccess) ph_collect(w);
    cudaGetLastError();
  }
  for (int ph = 0; ph < PH_COUNT; ++ph) {
    if (ms) ms[ph] = s->ph_ms[ph];
    if (launches) launches[ph] = s->ph_launches[ph];
  }
  return SV_OK;
}

uint64_t sv_launch_count(void) { return g_launches.load(); }

void sv_transfer_bytes(uint64_t* h2d, uint64_t* d2h) {
  if (h2d) *h2d = g_h2d.load();
  if (d2h) *d2h = g_d2h.load();
}

}  // extern "C"
