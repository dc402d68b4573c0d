// C ABI of the batched form (svb_*, declared in include/sv.h): many circuits,
// each a segment of one device-resident state, advanced one gate per circuit
// per step with per-circuit top-k truncation (Sec. III) after every step.
#include <algorithm>
#include <array>
#include <cstdio>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "batch.h"
#include "host_util.h"
#include "sv.h"

using namespace sv;

namespace {

enum SlotState { SLOT_FREE = 0, SLOT_USED = 1, SLOT_REMOVING = 2 };

struct Slot {
  int state = SLOT_FREE;
  int n = 0;
  uint64_t K = 0;
  uint64_t count = 0;   // terms of this segment
  uint64_t offset = 0;  // first term in the current buffers
  double F = 1.0;
  uint64_t count_ub = 0;  // upper bound of count while steps are in flight (one launch per step)
  uint64_t seq = 0;       // order of admission = order of the segments in the buffers
  uint8_t order[64];      // bit of qubit b in the sort order the segment is sorted by
};

// Peak readouts in flight (svb_peak_async): ring of result slots.
constexpr int PEAK_RING = 1024;

}  // namespace

struct svb_state {
  int prec = 0;
  cudaStream_t st = nullptr;
  sv_allocator alloc{};
  bool custom_alloc = false;
  size_t amp_bytes = 16;
  int max_slots = 0;
  std::vector<Slot> slots;

  uint64_t N = 0, cap = 0;
  uint64_t* keys[2] = {nullptr, nullptr};
  void* amps[2] = {nullptr, nullptr};
  uint64_t* probs[2] = {nullptr, nullptr};
  uint16_t* seg[2] = {nullptr, nullptr};
  int cur = 0;

  uint64_t sort_cap = 0;
  uint64_t* sk[2] = {nullptr, nullptr};
  uint32_t* sidx[2] = {nullptr, nullptr};
  uint32_t* heads = nullptr;
  uint64_t lb_entries = 0;
  uint64_t* lookback = nullptr;
  uint32_t* hist = nullptr;
  uint32_t* hist_host = nullptr;
  uint64_t* tile_counter = nullptr;

  SegGate* gates_dev = nullptr;
  SegGate* gates_host = nullptr;
  uint64_t* tables_dev = nullptr;  // [max_slots][SEG_TABLE_WORDS] per-slot sort-order tables
  uint16_t* rank_slot_dev = nullptr;   // [max_slots] slot of each segment rank (buffer order)
  uint16_t* rank_slot_host = nullptr;
  SegSel* sel_dev = nullptr;
  SegSel* sel_host = nullptr;
  uint32_t* sel_cnt = nullptr;
  uint64_t* sel_mass = nullptr;  // [max_slots][4]: total and before-bin mass (u128 each) of the collect scan
  uint64_t* sel_buf = nullptr;   // [max_slots][SEGSEL_CAP] (hi, lo) copies of a segment's cut bin
  uint32_t* sel_bufn = nullptr;
  uint64_t* bounds_dev = nullptr;   // [4][max_slots]: start, end of the mat-vec output; start, end after a cut
  uint64_t* bounds_host = nullptr;
  Ctl* ctl = nullptr;
  Ctl* ctl_host = nullptr;

  std::string err;
  bool broken = false;
  uint64_t steps = 0;

  // autotuner: per (kernel, precision, widest gate, size class) the launch
  // shape of each tuned kernel, chosen by timing every shape twice on live
  // steps of that class (any shape gives the same result)
  bool autotune = true;
  struct TuneEntry {
    std::vector<float> ms;  // [2 * shapes], -1 = not timed yet
    int best = -1;
  };
  std::map<uint64_t, TuneEntry> tune;
  uint64_t tune_trials = 0;
  cudaEvent_t tev[3][2] = {};

  // CUDA graphs of the two enqueued parts of a step, keyed by everything
  // that is baked into the launches (sizes, shapes, buffer parity and the
  // buffer generation, bumped by every reallocation)
  bool own_stream = false;
  bool graphs_on = true;
  uint64_t gen = 0;
  // the layer kernel: every step one persistent cooperative launch (with
  // the gate-table upload and the readback, one graph replay)
  bool layer_on = true;
  int sms = 0;
  int layer_per_sm[5] = {};     // most co-resident blocks per SM by grouping width m (0: not queried yet)
  // autotuning of the layer kernel's blocks per SM: a step's launch is timed
  // with events that are read when its table set is reused (two steps on)
  cudaEvent_t lev[2][2] = {};
  uint64_t lev_key[2] = {};
  int lev_cfg[2] = {}, lev_shapes[2] = {};
  bool lev_pending[2] = {};
  LayerStep* step_dev = nullptr;
  LayerStep* step_host = nullptr;
  LayerCtl* lc_dev = nullptr;
  LayerCtl* lc_host = nullptr;
  uint32_t* sel_cnt2 = nullptr;   // second parity of the select histograms
  uint64_t* sel_mass2 = nullptr;
  uint32_t* sel_bufn2 = nullptr;
  uint32_t* layer_part = nullptr;  // partition counts and offsets, merge splits
  uint64_t layer_part_words = 0;
  uint64_t* layer_lb = nullptr;    // look-backs of the heads, the mat-vec and the compaction
  uint64_t layer_lb_heads = 0, layer_lb_apply = 0, layer_lb_trunc = 0;
  uint64_t layer_launches = 0;
  // With one launch per step the steps run asynchronously: the device holds
  // the state's buffer set, term count, slot bounds and retained masses, the
  // host keeps upper bounds of the slot counts and reads the rest back
  // (b_settle) only when a call needs it.  The gate tables alternate between
  // two pinned buffer sets (tparity), each reused once the step that read it
  // has completed (upload_ev).
  bool pending = false;
  int tparity = 0;
  cudaEvent_t upload_ev[2] = {};
  double* F_dev = nullptr;     // [max_slots]
  double* F_mirror = nullptr;  // pinned [max_slots]
  uint64_t next_seq = 0;
  uint64_t* peak_part = nullptr;   // [PEAK_SEG_BLOCKS][2]
  uint64_t* ring_dev = nullptr;    // [PEAK_RING][4]
  uint64_t* ring_host = nullptr;   // pinned [PEAK_RING][4]: key, probability bits, mass bits, error bits
  cudaEvent_t ring_ev[PEAK_RING] = {};
  uint64_t ring_ticket[PEAK_RING] = {};  // ticket + 1 held by each ring slot (0: free)
  uint64_t next_ticket = 0;

  std::map<std::array<uint64_t, 12>, cudaGraphExec_t> graphs;
  std::set<std::array<uint64_t, 12>> seen_keys;  // keys enqueued once without a graph
  uint64_t graph_launches = 0, graph_captures = 0;
};

namespace {

sv_status b_settle(svb_state* b);

void* b_alloc(svb_state* b, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (b->custom_alloc) return b->alloc.alloc(bytes, b->alloc.ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void b_free(svb_state* b, void* p) {
  if (!p) return;
  if (b->custom_alloc) b->alloc.free(p, b->alloc.ctx);
  else cudaFree(p);
}

sv_status b_fail(svb_state* b, sv_status code, const std::string& msg) {
  b->err = msg;
  return code;
}

sv_status b_cuda(svb_state* b, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return SV_OK;
  b->broken = true;
  return b_fail(b, SV_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

sv_status b_sync_ctl(svb_state* b, const char* where) {
  cudaError_t e = cudaMemcpyAsync(b->ctl_host, b->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  sv_status rc = b_cuda(b, e, where);
  if (rc != SV_OK) return rc;
  if (b->ctl_host->err & ERR_TIMEOUT) {
    b->broken = true;
    return b_fail(b, SV_E_TIMEOUT, std::string(where) + ": a bounded device wait ran out");
  }
  if (b->ctl_host->err & (ERR_MASS | ERR_INVARIANT)) {
    b->broken = true;
    return b_fail(b, SV_E_STATE, std::string(where) + ": device state error");
  }
  return SV_OK;
}

sv_status b_lookback(svb_state* b, uint64_t entries) {
  if (entries <= b->lb_entries) return SV_OK;
  const uint64_t want = entries + entries / 2 + 1024;
  uint64_t* p = (uint64_t*)b_alloc(b, want * 8);
  if (!p) return b_fail(b, SV_E_NOMEM, "look-back buffer allocation failed");
  b_free(b, b->lookback);
  b->lookback = p;
  b->lb_entries = want;
  ++b->gen;
  return SV_OK;
}

// Buffers for `need` terms; the current contents are preserved.
sv_status b_state_cap(svb_state* b, uint64_t need) {
  if (need <= b->cap) return SV_OK;
  if (b->pending) {  // the copy below needs the exact state, and steps in flight use the old buffers
    sv_status rs = b_settle(b);
    if (rs != SV_OK) return rs;
  }
  uint64_t cap = b->cap * 2 > need ? b->cap * 2 : need;
  if (cap < 4096) cap = 4096;
  uint64_t* k[2];
  void* a[2];
  uint64_t* p[2];
  uint16_t* g[2];
  for (int i = 0; i < 2; ++i) {
    k[i] = (uint64_t*)b_alloc(b, cap * 8);
    a[i] = b_alloc(b, cap * b->amp_bytes);
    p[i] = (uint64_t*)b_alloc(b, cap * 8);
    g[i] = (uint16_t*)b_alloc(b, cap * 2);
    if (!k[i] || !a[i] || !p[i] || !g[i]) {
      for (int j = 0; j <= i; ++j) {
        b_free(b, k[j]);
        b_free(b, a[j]);
        b_free(b, p[j]);
        b_free(b, g[j]);
      }
      return b_fail(b, SV_E_NOMEM, "batch state allocation failed");
    }
  }
  if (b->N) {
    cudaMemcpyAsync(k[0], b->keys[b->cur], b->N * 8, cudaMemcpyDeviceToDevice, b->st);
    cudaMemcpyAsync(a[0], b->amps[b->cur], b->N * b->amp_bytes, cudaMemcpyDeviceToDevice, b->st);
    cudaMemcpyAsync(p[0], b->probs[b->cur], b->N * 8, cudaMemcpyDeviceToDevice, b->st);
    cudaMemcpyAsync(g[0], b->seg[b->cur], b->N * 2, cudaMemcpyDeviceToDevice, b->st);
  }
  sv_status rc = b_cuda(b, cudaStreamSynchronize(b->st), "batch state growth");
  for (int i = 0; i < 2; ++i) {
    b_free(b, b->keys[i]);
    b_free(b, b->amps[i]);
    b_free(b, b->probs[i]);
    b_free(b, b->seg[i]);
    b->keys[i] = k[i];
    b->amps[i] = a[i];
    b->probs[i] = p[i];
    b->seg[i] = g[i];
  }
  b->cur = 0;
  b->cap = cap;
  ++b->gen;
  if (rc == SV_OK && b->layer_on)  // the device bookkeeping follows the copy into buffer set 0
    rc = b_cuda(b, cudaMemsetAsync(&b->lc_dev->cur, 0, sizeof(uint32_t), b->st), "batch state growth");
  return rc;
}

sv_status b_sort_cap(svb_state* b, uint64_t need) {
  if (need > b->sort_cap) {
    uint64_t cap = b->sort_cap * 2 > need ? b->sort_cap * 2 : need;
    if (cap < 4096) cap = 4096;
    for (int i = 0; i < 2; ++i) {
      b_free(b, b->sk[i]);
      b_free(b, b->sidx[i]);
      b->sk[i] = (uint64_t*)b_alloc(b, cap * 8);
      b->sidx[i] = (uint32_t*)b_alloc(b, cap * 4);
    }
    b_free(b, b->heads);
    b->heads = (uint32_t*)b_alloc(b, cap * 4);
    if (!b->sk[0] || !b->sk[1] || !b->sidx[0] || !b->sidx[1] || !b->heads) {
      b->sort_cap = 0;
      return b_fail(b, SV_E_NOMEM, "batch sort buffer allocation failed");
    }
    b->sort_cap = cap;
    ++b->gen;
  }
  return b_lookback(b, sort_tiles(need) * RADIX + 16);
}

// Scratch of the layer kernel for N terms in (nkeep of them in slots that
// stay) and gates of up to 2^mmax outputs per group.
// Whether that scratch must grow first.
bool layer_grows(const svb_state* b, uint64_t N, uint64_t nkeep, int mmax) {
  return 2 * 16 * (N / 4096 + 2) + 64 > b->layer_part_words || nkeep / 4096 + 2 > b->layer_lb_heads ||
         nkeep / 256 + 2 > b->layer_lb_apply || (nkeep << mmax) / 2048 + 2 > b->layer_lb_trunc;
}

sv_status b_layer_cap(svb_state* b, uint64_t N, uint64_t nkeep, int mmax) {
  const uint64_t tiles = N / 4096 + 2;
  const uint64_t part = 2 * 16 * tiles + 64;
  if (part > b->layer_part_words) {
    const uint64_t want = part + part / 2;
    uint32_t* p = (uint32_t*)b_alloc(b, want * 4);
    if (!p) return b_fail(b, SV_E_NOMEM, "layer scratch allocation failed");
    b_free(b, b->layer_part);
    b->layer_part = p;
    b->layer_part_words = want;
    ++b->gen;
  }
  const uint64_t heads = nkeep / 4096 + 2, apply = nkeep / 256 + 2, trunc = (nkeep << mmax) / 2048 + 2;
  if (heads > b->layer_lb_heads || apply > b->layer_lb_apply || trunc > b->layer_lb_trunc) {
    const uint64_t h = std::max(heads + heads / 2, b->layer_lb_heads), a = std::max(apply + apply / 2, b->layer_lb_apply),
                   t = std::max(trunc + trunc / 2, b->layer_lb_trunc);
    uint64_t* p = (uint64_t*)b_alloc(b, (h + a + t) * 8);
    if (!p) return b_fail(b, SV_E_NOMEM, "layer look-back allocation failed");
    b_free(b, b->layer_lb);
    b->layer_lb = p;
    b->layer_lb_heads = h;
    b->layer_lb_apply = a;
    b->layer_lb_trunc = t;
    ++b->gen;
  }
  return SV_OK;
}

enum TuneKernel { TK_APPLY = 0, TK_SELECT = 1, TK_TRUNC = 2, TK_LAYER = 3 };

uint64_t tune_key(int kernel, int prec, int mmax, uint64_t n) {
  const int sclass = n ? 63 - __builtin_clzll(n) : 0;
  return ((uint64_t)kernel << 24) | ((uint64_t)prec << 16) | ((uint64_t)mmax << 8) | (uint64_t)sclass;
}

// The shape to run: the first one not yet timed twice, else the fastest.
int tune_pick(svb_state* b, uint64_t key, int shapes, int dflt) {
  if (!b->autotune || shapes <= 1) return dflt;
  svb_state::TuneEntry& e = b->tune[key];
  if (e.ms.empty()) e.ms.assign(2 * shapes, -1.f);
  for (int i = 0; i < 2 * shapes; ++i)
    if (e.ms[i] < 0.f) return i % shapes;
  if (e.best < 0) {
    float best = 0.f;
    for (int c = 0; c < shapes; ++c) {
      const float t = std::min(e.ms[c], e.ms[c + shapes]);
      if (e.best < 0 || t < best) {
        e.best = c;
        best = t;
      }
    }
  }
  return e.best;
}

bool tune_settled(svb_state* b, uint64_t key, int shapes) {
  if (!b->autotune || shapes <= 1) return true;
  auto it = b->tune.find(key);
  if (it == b->tune.end() || it->second.ms.empty()) return false;
  for (float t : it->second.ms)
    if (t < 0.f) return false;
  return true;
}

void drop_graphs(svb_state* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

// Enqueue one part of a step: replay its graph when one was captured under
// the same key, capture it when the key comes a second time, else (a key
// seen once, or graphs off or unavailable) enqueue the launches directly.
// Keys that never repeat (term counts change while states grow and
// circuits retire) so cost no capture and instantiation.
template <typename F>
sv_status run_part(svb_state* b, bool use_graph, const std::array<uint64_t, 12>& key, F&& enqueue) {
  if (!(use_graph && b->graphs_on)) return enqueue();
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    if (b->seen_keys.insert(key).second) {
      if (b->seen_keys.size() > 4096) {
        b->seen_keys.clear();
        b->seen_keys.insert(key);
      }
      return enqueue();
    }
    if (b->graphs.size() >= 64) drop_graphs(b);
    if (cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      b->graphs_on = false;
      return enqueue();
    }
    const sv_status rc = enqueue();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->st, &g);
    cudaGraphExec_t x = nullptr;
    if (rc != SV_OK || e != cudaSuccess || cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      b->graphs_on = false;  // run this and later steps without graphs (nothing captured has run)
      return enqueue();
    }
    cudaGraphDestroy(g);
    it = b->graphs.emplace(key, x).first;
    ++b->graph_captures;
  }
  ++b->graph_launches;
  if (cudaGraphLaunch(it->second, b->st) != cudaSuccess) {
    cudaGetLastError();
    return b_fail(b, SV_E_CUDA, "svb_step: graph launch failed");
  }
  return SV_OK;
}

// Wait for the stream and check the control block read back with it.
sv_status b_wait(svb_state* b, const char* where) {
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  sv_status rc = b_cuda(b, e, where);
  if (rc != SV_OK) return rc;
  if (b->ctl_host->err & ERR_TIMEOUT) {
    b->broken = true;
    return b_fail(b, SV_E_TIMEOUT, std::string(where) + ": a bounded device wait ran out");
  }
  if (b->ctl_host->err & (ERR_MASS | ERR_INVARIANT)) {
    b->broken = true;
    return b_fail(b, SV_E_STATE, std::string(where) + ": device state error");
  }
  return SV_OK;
}

// Bring the host's view of the state up to date after asynchronous steps:
// wait for the stream, read the device bookkeeping (buffer set, term count,
// slot bounds, retained masses, error bits) and set every slot's offset,
// count and mass from it.
sv_status b_settle(svb_state* b) {
  if (!b->pending) return SV_OK;
  cudaMemcpyAsync(b->lc_host, b->lc_dev, sizeof(LayerCtl), cudaMemcpyDeviceToHost, b->st);
  cudaMemcpyAsync(b->ctl_host, b->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, b->st);
  cudaMemcpyAsync(b->bounds_host, b->bounds_dev, sizeof(uint64_t) * 4 * b->max_slots, cudaMemcpyDeviceToHost, b->st);
  cudaMemcpyAsync(b->F_mirror, b->F_dev, sizeof(double) * b->max_slots, cudaMemcpyDeviceToHost, b->st);
  sv_status rc = b_wait(b, "batch readback");
  if (rc != SV_OK) return rc;
  if (b->lc_host->unresolved) {
    b->broken = true;
    return b_fail(b, SV_E_STATE, "svb_step: segmented select did not resolve");
  }
  b->cur = (int)b->lc_host->cur;
  b->N = b->lc_host->n_cur;
  const uint64_t* bh = b->bounds_host + (b->lc_host->truncated ? 2 * b->max_slots : 0);
  for (int s = 0; s < b->max_slots; ++s) {
    Slot& sl = b->slots[s];
    if (sl.state == SLOT_FREE) continue;
    const uint64_t a = bh[s], e = bh[b->max_slots + s];
    sl.offset = e > a ? a : 0;  // a slot with no terms keeps start all ones
    sl.count = e > a ? e - a : 0;
    sl.count_ub = sl.count;
    sl.F = b->F_mirror[s];
  }
  b->pending = false;
  return SV_OK;
}

void tune_record(svb_state* b, uint64_t key, int shapes, int shape, float ms) {
  if (!b->autotune || shapes <= 1) return;
  svb_state::TuneEntry& e = b->tune[key];
  for (int i = 0; i < (int)e.ms.size(); ++i)
    if (e.ms[i] < 0.f && i % shapes == shape) {
      e.ms[i] = ms;
      ++b->tune_trials;
      return;
    }
}

#define SVB_GUARD(b)                                                                                   \
  do {                                                                                                 \
    if (!(b)) return SV_E_ARG;                                                                         \
    if ((b)->broken) return b_fail((b), SV_E_STATE, "batch handle unusable after an earlier failure: " + (b)->err); \
  } while (0)

}  // namespace

// The step as separate kernels (two enqueued parts, each replayed as a CUDA
// graph once its shapes are settled, and a host wait after each).
static sv_status step_kernels(svb_state* b, int top, uint64_t N, uint64_t nkeep, int shift, int nbits, int mmax,
                       bool may_truncate, bool& truncated) {
  sv_status rc = SV_OK;
  const uint64_t apply_tiles = nkeep / 256 + 2;  // one group per thread: the most tiles of any shape
  if (rc == SV_OK) rc = b_lookback(b, apply_tiles + 16);
  if (rc != SV_OK) return rc;
  const uint64_t n_cand = nkeep << mmax;  // the most candidates the mat-vec can emit
  if (may_truncate) rc = b_lookback(b, std::max(apply_tiles, n_cand / 2048 + 2) + 16);
  if (rc != SV_OK) return rc;
  // The step is enqueued with device-side term counts in two parts (each
  // replayed as a CUDA graph once its shapes are settled); the host waits
  // after each: to confirm every segment's cut is resolved, and for the new
  // counts.
  const int alt = 1 - b->cur;
  uint64_t* start_dev = b->bounds_dev;
  uint64_t* end_dev = b->bounds_dev + b->max_slots;
  uint64_t* start_tr = b->bounds_dev + 2 * b->max_slots;
  uint64_t* end_tr = b->bounds_dev + 3 * b->max_slots;
  const uint64_t key_apply = tune_key(TK_APPLY, b->prec, mmax, nkeep);
  const uint64_t key_sel = tune_key(TK_SELECT, b->prec, mmax, n_cand);
  const uint64_t key_trunc = tune_key(TK_TRUNC, b->prec, mmax, n_cand);
  const int n_apply = seg_apply_configs(mmax);
  const int cfg_apply = tune_pick(b, key_apply, n_apply, mmax == 2 ? 1 : 0);
  const int cfg_sel = may_truncate ? tune_pick(b, key_sel, SEGSEL_CONFIGS, 1) : -1;
  const int cfg_trunc = may_truncate ? tune_pick(b, key_trunc, SEGTRUNC_CONFIGS, 1) : -1;
  const bool settled = tune_settled(b, key_apply, n_apply) &&
                       (!may_truncate || (tune_settled(b, key_sel, SEGSEL_CONFIGS) &&
                                          tune_settled(b, key_trunc, SEGTRUNC_CONFIGS)));
  const bool timing = b->autotune && !settled;  // events only while shapes are explored
  std::array<uint64_t, 12> key_a = {0, N, nkeep, (uint64_t)top, (uint64_t)shift, (uint64_t)nbits, (uint64_t)mmax,
                                    (uint64_t)cfg_apply, (uint64_t)(cfg_sel + 1), (uint64_t)b->cur, b->gen,
                                    (uint64_t)may_truncate};
  rc = run_part(b, settled, key_a, [&]() -> sv_status {
    cudaMemcpyAsync(b->gates_dev, b->gates_host, sizeof(SegGate) * top, cudaMemcpyHostToDevice, b->st);
    cudaMemcpyAsync(b->rank_slot_dev, b->rank_slot_host, sizeof(uint16_t) * top, cudaMemcpyHostToDevice, b->st);
    // grouping: every segment is sorted by its previous order, so the terms
    // with equal low M bits of the new sort key are already sorted by it: a
    // stable partition by those bits and M merge levels sort the batch
    launch_seg_tables(b->gates_dev, top, b->tables_dev, b->st);
    launch_seg_keys(b->keys[b->cur], b->seg[b->cur], N, b->gates_dev, b->tables_dev, shift, b->sk[1], b->st);
    cudaMemsetAsync(b->hist, 0, sizeof(uint32_t) * 16, b->st);  // the partition's run totals
    SortScratch sc;
    sc.hist = b->hist;
    sc.hist_host = nullptr;
    sc.lookback = b->lookback;
    sc.lookback_tiles = b->lb_entries / RADIX;
    sc.tile_counter = b->tile_counter;
    sc.err = &b->ctl->err;
    GateParams gp;
    std::memset(&gp, 0, sizeof(gp));
    gp.m = mmax > 1 ? mmax : 1;
    gp.direct = 1;
    cudaError_t ce;
    int nl = 0;
    const int w = regroup_terms(b->sk[1], N, gp, b->sk, b->sidx, sc, b->st, &nl, &ce);
    if (ce != cudaSuccess) return b_cuda(b, ce, "svb_step grouping");
    launch_seg_heads(b->sk[w], nkeep, shift, b->gates_dev, b->rank_slot_dev, b->heads, b->lookback, b->ctl, b->st);
    // the mat-vec counts the select's first digit per slot when a cut may
    // follow, and records where each slot's outputs start and end
    if (may_truncate) cudaMemsetAsync(b->sel_cnt, 0, sizeof(uint32_t) * SEL_BINS * top, b->st);
    cudaMemsetAsync(start_dev, 0xff, sizeof(uint64_t) * b->max_slots, b->st);
    cudaMemsetAsync(end_dev, 0, sizeof(uint64_t) * b->max_slots, b->st);
    if (timing) cudaEventRecord(b->tev[TK_APPLY][0], b->st);
    launch_seg_apply(b->prec, b->sk[w], b->sidx[w], nkeep, b->heads, b->amps[b->cur], shift, mmax, b->gates_dev,
                     b->rank_slot_dev, b->keys[b->cur],
                     b->keys[alt], b->amps[alt], b->probs[alt], b->seg[alt], may_truncate ? b->sel_cnt : nullptr,
                     start_dev, end_dev, b->lookback, b->ctl, apply_tiles, cfg_apply, b->st);
    if (timing) cudaEventRecord(b->tev[TK_APPLY][1], b->st);
    if (may_truncate) {
      // per-segment top-k: three levels normally resolve every cut
      // (exponent bin, top mantissa bin, the copied bin); the first one's
      // histogram came with the mat-vec, so two scans follow its pick
      launch_segsel_init(b->sel_dev, b->gates_dev, start_dev, end_dev, top, b->st);
      if (timing) cudaEventRecord(b->tev[TK_SELECT][0], b->st);
      launch_segsel_pick(b->sel_dev, top, b->sel_cnt, b->st);
      for (int level = 1; level < 3; ++level) {
        launch_segsel_level(b->probs[alt], b->keys[alt], b->seg[alt], &b->ctl->count[1], b->sel_dev, top, b->sel_cnt,
                            b->sel_mass, b->sel_buf, b->sel_bufn, &b->ctl->err, cfg_sel, b->st);
        launch_segsel_finish(b->sel_buf, b->sel_bufn, b->sel_mass, b->sel_dev, top, &b->ctl->err, b->st);
      }
      if (timing) cudaEventRecord(b->tev[TK_SELECT][1], b->st);
      cudaMemcpyAsync(b->sel_host, b->sel_dev, sizeof(SegSel) * top, cudaMemcpyDeviceToHost, b->st);
    } else {
      cudaMemcpyAsync(b->bounds_host, b->bounds_dev, sizeof(uint64_t) * 4 * b->max_slots, cudaMemcpyDeviceToHost,
                      b->st);
    }
    cudaMemcpyAsync(b->ctl_host, b->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, b->st);
    return SV_OK;
  });
  if (rc != SV_OK) return rc;
  rc = b_wait(b, "svb_step");
  if (rc != SV_OK) return rc;
  for (int s = 0; s < b->max_slots; ++s)
    if (b->slots[s].state == SLOT_REMOVING) b->slots[s] = Slot();
  b->cur = alt;
  if (may_truncate) {
    // rarely a cut needs more levels (long runs of equal probabilities)
    bool all_done = false;
    for (int extra = 0;; ++extra) {
      all_done = true;
      for (int s = 0; s < top; ++s)
        if (b->sel_host[s].active && !b->sel_host[s].done) all_done = false;
      if (all_done || extra >= 13) break;
      launch_segsel_level(b->probs[b->cur], b->keys[b->cur], b->seg[b->cur], &b->ctl->count[1], b->sel_dev, top,
                          b->sel_cnt, b->sel_mass, b->sel_buf, b->sel_bufn, &b->ctl->err, cfg_sel, b->st);
      launch_segsel_finish(b->sel_buf, b->sel_bufn, b->sel_mass, b->sel_dev, top, &b->ctl->err, b->st);
      cudaMemcpyAsync(b->sel_host, b->sel_dev, sizeof(SegSel) * top, cudaMemcpyDeviceToHost, b->st);
      rc = b_sync_ctl(b, "svb_step select");
      if (rc != SV_OK) return rc;
    }
    if (!all_done) {
      b->broken = true;
      return b_fail(b, SV_E_STATE, "svb_step: segmented select did not resolve");
    }
    for (int s = 0; s < top; ++s)
      if (b->sel_host[s].active && b->sel_host[s].done == 1) truncated = true;
    const int alt2 = 1 - b->cur;
    std::array<uint64_t, 12> key_b = {1, N, nkeep, (uint64_t)top, n_cand, (uint64_t)truncated, (uint64_t)mmax,
                                      (uint64_t)cfg_trunc, 0, (uint64_t)b->cur, b->gen, 0};
    rc = run_part(b, settled, key_b, [&]() -> sv_status {
      if (truncated) {
        launch_segsel_scale(b->sel_dev, top, b->st);
        cudaMemsetAsync(start_tr, 0xff, sizeof(uint64_t) * b->max_slots, b->st);
        cudaMemsetAsync(end_tr, 0, sizeof(uint64_t) * b->max_slots, b->st);
        if (timing) cudaEventRecord(b->tev[TK_TRUNC][0], b->st);
        launch_seg_truncate(b->prec, b->keys[b->cur], b->amps[b->cur], b->probs[b->cur], b->seg[b->cur],
                            &b->ctl->count[1], n_cand, b->sel_dev, b->keys[alt2], b->amps[alt2], b->seg[alt2],
                            start_tr, end_tr, b->lookback, b->ctl, cfg_trunc, b->st);
        if (timing) cudaEventRecord(b->tev[TK_TRUNC][1], b->st);
      }
      cudaMemcpyAsync(b->bounds_host, b->bounds_dev, sizeof(uint64_t) * 4 * b->max_slots, cudaMemcpyDeviceToHost,
                      b->st);
      cudaMemcpyAsync(b->ctl_host, b->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, b->st);
      return SV_OK;
    });
    if (rc != SV_OK) return rc;
    rc = b_wait(b, "svb_step truncate");
    if (rc != SV_OK) return rc;
    if (truncated) b->cur = alt2;
  }
  b->N = truncated ? b->ctl_host->count[2] : b->ctl_host->count[1];
  if (timing) {  // the stream is idle: every recorded interval is complete
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->tev[TK_APPLY][0], b->tev[TK_APPLY][1]) == cudaSuccess)
      tune_record(b, key_apply, n_apply, cfg_apply, ms);
    if (cfg_sel >= 0 && cudaEventElapsedTime(&ms, b->tev[TK_SELECT][0], b->tev[TK_SELECT][1]) == cudaSuccess)
      tune_record(b, key_sel, SEGSEL_CONFIGS, cfg_sel, ms);
    if (truncated && cudaEventElapsedTime(&ms, b->tev[TK_TRUNC][0], b->tev[TK_TRUNC][1]) == cudaSuccess)
      tune_record(b, key_trunc, SEGTRUNC_CONFIGS, cfg_trunc, ms);
    cudaGetLastError();
  }
  return SV_OK;
}

// The step as one persistent launch of the layer kernel: the gate-table
// upload, the launch (one graph replay once the shape recurs) and no wait;
// the term counts stay on the device.
static sv_status step_layer(svb_state* b, int par, int top, uint64_t N, uint64_t nkeep, int shift, int mmax) {
  const int m = mmax > 1 ? mmax : 1;
  sv_status rc = b_layer_cap(b, N, nkeep, m);
  if (rc != SV_OK) return rc;
  if (!b->layer_per_sm[m]) {
    unsigned g = 0;
    rc = b_cuda(b, seg_layer_grid(b->prec, m, b->sms, &g), "svb_step layer occupancy");
    if (rc != SV_OK) return rc;
    b->layer_per_sm[m] = (int)(g / (unsigned)b->sms);
  }
  // blocks per SM: the most that fit, or one fewer (more shared memory and
  // cache per block), chosen by timing live steps of each class (term
  // counts by factors of 4: few classes, so little of a run goes to trials)
  const int most = b->layer_per_sm[m];
  const int shapes = most < 2 ? most : 2;
  const uint64_t tkey = tune_key(TK_LAYER, b->prec, m, N ? 1ull << ((63 - __builtin_clzll(N)) & ~1) : 0);
  const int cfg = tune_pick(b, tkey, shapes, 0);
  const bool timing = b->autotune && !tune_settled(b, tkey, shapes);
  const unsigned grid = (unsigned)((most - cfg) * b->sms);
  LayerStep* sh = b->step_host + par;
  sh->shift = shift;
  sh->top = top;
  sh->m = m;
  sh->pad = 0;
  SegGate* gh = b->gates_host + (size_t)par * b->max_slots;
  uint16_t* rh = b->rank_slot_host + (size_t)par * b->max_slots;
  LayerParams P;
  std::memset(&P, 0, sizeof(P));
  P.step = b->step_dev;
  P.lc = b->lc_dev;
  P.ctl = b->ctl;
  for (int i = 0; i < 2; ++i) {
    P.keys[i] = b->keys[i];
    P.amps[i] = b->amps[i];
    P.probs[i] = b->probs[i];
    P.seg[i] = b->seg[i];
    P.sk[i] = b->sk[i];
    P.sidx[i] = b->sidx[i];
  }
  P.F = b->F_dev;
  P.heads = b->heads;
  P.hist16 = b->hist;
  P.part = b->layer_part;
  P.lb = b->layer_lb;
  P.lb_heads_words = b->layer_lb_heads;
  P.lb_apply_words = b->layer_lb_apply;
  P.lb_trunc_words = b->layer_lb_trunc;
  P.gates = b->gates_dev;
  P.rank_slot = b->rank_slot_dev;
  P.tables = b->tables_dev;
  P.sel = b->sel_dev;
  P.sel_cnt[0] = b->sel_cnt;
  P.sel_cnt[1] = b->sel_cnt2;
  P.sel_mass[0] = b->sel_mass;
  P.sel_mass[1] = b->sel_mass2;
  P.sel_buf = b->sel_buf;
  P.sel_bufn[0] = b->sel_bufn;
  P.sel_bufn[1] = b->sel_bufn2;
  P.start = b->bounds_dev;
  P.end = b->bounds_dev + b->max_slots;
  P.start_tr = b->bounds_dev + 2 * b->max_slots;
  P.end_tr = b->bounds_dev + 3 * b->max_slots;
  const std::array<uint64_t, 12> key = {2, (uint64_t)top, (uint64_t)m, (uint64_t)par, b->gen, grid, 0, 0, 0, 0, 0, 0};
  if (timing) cudaEventRecord(b->lev[par][0], b->st);
  rc = run_part(b, true, key, [&]() -> sv_status {
    cudaMemcpyAsync(b->gates_dev, gh, sizeof(SegGate) * top, cudaMemcpyHostToDevice, b->st);
    cudaMemcpyAsync(b->rank_slot_dev, rh, sizeof(uint16_t) * top, cudaMemcpyHostToDevice, b->st);
    cudaMemcpyAsync(b->step_dev, sh, sizeof(LayerStep), cudaMemcpyHostToDevice, b->st);
    const cudaError_t e = launch_seg_layer(b->prec, m, P, grid, b->st);
    if (e != cudaSuccess) return b_cuda(b, e, "svb_step layer launch");
    return SV_OK;
  });
  if (rc != SV_OK) return rc;
  if (timing) {
    cudaEventRecord(b->lev[par][1], b->st);
    b->lev_key[par] = tkey;
    b->lev_cfg[par] = cfg;
    b->lev_shapes[par] = shapes;
    b->lev_pending[par] = true;
  }
  rc = b_cuda(b, cudaEventRecord(b->upload_ev[par], b->st), "svb_step");
  if (rc != SV_OK) return rc;
  b->pending = true;
  ++b->layer_launches;
  return SV_OK;
}

extern "C" {

sv_status svb_destroy(svb_state* b);

sv_status svb_create(int max_slots, int prec, void* cuda_stream, const sv_allocator* alloc, svb_state** out) {
  if (!out) return SV_E_ARG;
  *out = nullptr;
  if (max_slots < 1 || max_slots > 1023 || (prec != SV_C128 && prec != SV_C64)) return SV_E_ARG;
  if (alloc && (!alloc->alloc || !alloc->free)) return SV_E_ARG;
  if (batch_prepare() != cudaSuccess) {  // kernel attributes of this device, before any capture
    cudaGetLastError();
    return SV_E_CUDA;
  }
  svb_state* b = new svb_state();
  b->prec = prec;
  b->st = (cudaStream_t)cuda_stream;
  if (!b->st) {  // a stream of its own: the legacy default stream cannot be captured into graphs
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      b->st = nullptr;
    } else {
      b->own_stream = true;
    }
  }
  b->amp_bytes = prec == SV_C128 ? 16 : 8;
  b->max_slots = max_slots;
  b->slots.resize(max_slots);
  if (alloc) {
    b->alloc = *alloc;
    b->custom_alloc = true;
  }
  sv_status rc = SV_OK;
  b->hist = (uint32_t*)b_alloc(b, sizeof(uint32_t) * MAX_PASSES * RADIX);
  b->tile_counter = (uint64_t*)b_alloc(b, 256);
  b->ctl = (Ctl*)b_alloc(b, sizeof(Ctl));
  b->gates_dev = (SegGate*)b_alloc(b, sizeof(SegGate) * max_slots);
  b->tables_dev = (uint64_t*)b_alloc(b, sizeof(uint64_t) * SEG_TABLE_WORDS * max_slots);
  b->rank_slot_dev = (uint16_t*)b_alloc(b, sizeof(uint16_t) * max_slots);
  b->sel_dev = (SegSel*)b_alloc(b, sizeof(SegSel) * max_slots);
  b->sel_cnt = (uint32_t*)b_alloc(b, sizeof(uint32_t) * SEL_BINS * max_slots);
  b->sel_mass = (uint64_t*)b_alloc(b, sizeof(uint64_t) * 4 * max_slots);
  b->sel_buf = (uint64_t*)b_alloc(b, sizeof(uint64_t) * 2 * SEGSEL_CAP * max_slots);
  b->sel_bufn = (uint32_t*)b_alloc(b, sizeof(uint32_t) * max_slots);
  b->bounds_dev = (uint64_t*)b_alloc(b, sizeof(uint64_t) * 4 * max_slots);
  b->sel_cnt2 = (uint32_t*)b_alloc(b, sizeof(uint32_t) * SEL_BINS * max_slots);
  b->sel_mass2 = (uint64_t*)b_alloc(b, sizeof(uint64_t) * 4 * max_slots);
  b->sel_bufn2 = (uint32_t*)b_alloc(b, sizeof(uint32_t) * max_slots);
  b->step_dev = (LayerStep*)b_alloc(b, sizeof(LayerStep));
  b->lc_dev = (LayerCtl*)b_alloc(b, sizeof(LayerCtl));
  b->F_dev = (double*)b_alloc(b, sizeof(double) * max_slots);
  b->peak_part = (uint64_t*)b_alloc(b, sizeof(uint64_t) * 2 * PEAK_SEG_BLOCKS);
  b->ring_dev = (uint64_t*)b_alloc(b, sizeof(uint64_t) * 4 * PEAK_RING);
  if (!b->sel_cnt2 || !b->sel_mass2 || !b->sel_bufn2 || !b->step_dev || !b->lc_dev || !b->F_dev || !b->peak_part ||
      !b->ring_dev)
    rc = SV_E_NOMEM;
  if (!b->hist || !b->tile_counter || !b->ctl || !b->gates_dev || !b->tables_dev || !b->rank_slot_dev ||
      !b->sel_dev || !b->sel_cnt ||
      !b->sel_mass ||
      !b->sel_buf || !b->sel_bufn || !b->bounds_dev)
    rc = SV_E_NOMEM;
  if (rc == SV_OK && (cudaMallocHost(&b->hist_host, sizeof(uint32_t) * MAX_PASSES * RADIX) != cudaSuccess ||
                      cudaMallocHost(&b->ctl_host, sizeof(Ctl)) != cudaSuccess ||
                      cudaMallocHost(&b->gates_host, sizeof(SegGate) * 2 * max_slots) != cudaSuccess ||
                      cudaMallocHost(&b->rank_slot_host, sizeof(uint16_t) * 2 * max_slots) != cudaSuccess ||
                      cudaMallocHost(&b->sel_host, sizeof(SegSel) * max_slots) != cudaSuccess ||
                      cudaMallocHost(&b->bounds_host, sizeof(uint64_t) * 4 * max_slots) != cudaSuccess ||
                      cudaMallocHost(&b->step_host, sizeof(LayerStep) * 2) != cudaSuccess ||
                      cudaMallocHost(&b->lc_host, sizeof(LayerCtl)) != cudaSuccess ||
                      cudaMallocHost(&b->F_mirror, sizeof(double) * max_slots) != cudaSuccess ||
                      cudaMallocHost(&b->ring_host, sizeof(uint64_t) * 4 * PEAK_RING) != cudaSuccess))
    rc = SV_E_CUDA;
  for (int j = 0; j < 2 && rc == SV_OK; ++j)
    if (cudaEventCreateWithFlags(&b->upload_ev[j], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&b->lev[j][0]) != cudaSuccess || cudaEventCreate(&b->lev[j][1]) != cudaSuccess)
      rc = SV_E_CUDA;
  for (int j = 0; j < PEAK_RING && rc == SV_OK; ++j)
    if (cudaEventCreateWithFlags(&b->ring_ev[j], cudaEventDisableTiming) != cudaSuccess) rc = SV_E_CUDA;
  if (rc == SV_OK) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      rc = SV_E_CUDA;
  }
  for (int k = 0; k < 3 && rc == SV_OK; ++k)
    for (int j = 0; j < 2 && rc == SV_OK; ++j)
      if (cudaEventCreate(&b->tev[k][j]) != cudaSuccess) rc = SV_E_CUDA;
  if (rc == SV_OK) rc = b_state_cap(b, 4096);
  if (rc == SV_OK) rc = b_sort_cap(b, 4096);
  if (rc == SV_OK) rc = b_cuda(b, cudaMemsetAsync(b->ctl, 0, sizeof(Ctl), b->st), "svb_create");
  if (rc == SV_OK) rc = b_cuda(b, cudaMemsetAsync(b->lc_dev, 0, sizeof(LayerCtl), b->st), "svb_create");
  if (rc == SV_OK) std::memset(b->lc_host, 0, sizeof(LayerCtl));
  if (rc == SV_OK) rc = b_cuda(b, cudaStreamSynchronize(b->st), "svb_create");
  if (rc != SV_OK) {
    svb_destroy(b);
    return rc;
  }
  *out = b;
  return SV_OK;
}

sv_status svb_destroy(svb_state* b) {
  if (!b) return SV_OK;
  if (b->st) cudaStreamSynchronize(b->st);
  else cudaDeviceSynchronize();
  for (int i = 0; i < 2; ++i) {
    b_free(b, b->keys[i]);
    b_free(b, b->amps[i]);
    b_free(b, b->probs[i]);
    b_free(b, b->seg[i]);
    b_free(b, b->sk[i]);
    b_free(b, b->sidx[i]);
  }
  b_free(b, b->heads);
  b_free(b, b->lookback);
  b_free(b, b->hist);
  b_free(b, b->tile_counter);
  b_free(b, b->ctl);
  b_free(b, b->gates_dev);
  b_free(b, b->tables_dev);
  b_free(b, b->rank_slot_dev);
  b_free(b, b->sel_dev);
  b_free(b, b->sel_cnt);
  b_free(b, b->sel_mass);
  b_free(b, b->sel_buf);
  b_free(b, b->sel_bufn);
  b_free(b, b->bounds_dev);
  b_free(b, b->sel_cnt2);
  b_free(b, b->sel_mass2);
  b_free(b, b->sel_bufn2);
  b_free(b, b->step_dev);
  b_free(b, b->lc_dev);
  b_free(b, b->layer_part);
  b_free(b, b->layer_lb);
  b_free(b, b->F_dev);
  b_free(b, b->peak_part);
  b_free(b, b->ring_dev);
  for (int j = 0; j < 2; ++j) {
    if (b->upload_ev[j]) cudaEventDestroy(b->upload_ev[j]);
    for (int k = 0; k < 2; ++k)
      if (b->lev[j][k]) cudaEventDestroy(b->lev[j][k]);
  }
  for (int j = 0; j < PEAK_RING; ++j)
    if (b->ring_ev[j]) cudaEventDestroy(b->ring_ev[j]);
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 2; ++j)
      if (b->tev[k][j]) cudaEventDestroy(b->tev[k][j]);
  drop_graphs(b);
  if (b->own_stream) cudaStreamDestroy(b->st);
  if (b->hist_host) cudaFreeHost(b->hist_host);
  if (b->ctl_host) cudaFreeHost(b->ctl_host);
  if (b->gates_host) cudaFreeHost(b->gates_host);
  if (b->rank_slot_host) cudaFreeHost(b->rank_slot_host);
  if (b->sel_host) cudaFreeHost(b->sel_host);
  if (b->bounds_host) cudaFreeHost(b->bounds_host);
  if (b->step_host) cudaFreeHost(b->step_host);
  if (b->lc_host) cudaFreeHost(b->lc_host);
  if (b->F_mirror) cudaFreeHost(b->F_mirror);
  if (b->ring_host) cudaFreeHost(b->ring_host);
  delete b;
  return SV_OK;
}

sv_status svb_add(svb_state* b, int n, uint64_t K, double p, int* slot) {
  SVB_GUARD(b);
  if (!slot || n < 1 || n > 63 || K < 1) return b_fail(b, SV_E_ARG, "svb_add: n must be 1..63 and K >= 1");
  if (!(p >= 1.0)) return b_fail(b, SV_E_ARG, "svb_add: the batched form truncates by top-k only (p must be 1)");
  int s = -1, top = 0, maxn = n;
  for (int i = 0; i < b->max_slots; ++i) {
    const Slot& sl = b->slots[i];
    if (sl.state == SLOT_FREE) {
      if (s < 0) s = i;
      continue;
    }
    top = i + 1;
    if (sl.state == SLOT_USED && sl.n > maxn) maxn = sl.n;
  }
  if (s < 0) return b_fail(b, SV_E_ARG, "svb_add: no free slot");
  if (s + 1 > top) top = s + 1;
  int segbits = 0;
  while ((1 << segbits) <= top) ++segbits;
  if (maxn + segbits > 64)
    return b_fail(b, SV_E_ARG, "svb_add: the largest n plus the slot-index bits exceed the 64-bit sort key");
  Slot& sl = b->slots[s];
  if (b->layer_on) {  // appended at the end of the device-held state, no wait
    uint64_t total = 0;
    for (const Slot& o : b->slots) total += o.state == SLOT_FREE ? 0 : o.count_ub;
    sv_status rc = b_state_cap(b, total + 1);
    if (rc != SV_OK) return rc;
    launch_seg_append_layer(b->keys, b->amps, b->probs, b->seg, b->lc_dev, b->bounds_dev, b->max_slots, b->F_dev, s,
                            b->prec, b->st);
    rc = b_cuda(b, cudaGetLastError(), "svb_add");
    if (rc != SV_OK) return rc;
    b->pending = true;
  } else {
    sv_status rc = b_state_cap(b, b->N + 1);
    if (rc != SV_OK) return rc;
    launch_seg_append(b->keys[b->cur], b->amps[b->cur], b->probs[b->cur], b->seg[b->cur], b->N, s, b->prec, b->st);
    rc = b_cuda(b, cudaGetLastError(), "svb_add");
    if (rc != SV_OK) return rc;
    sl.offset = b->N;
    b->N += 1;
  }
  sl.state = SLOT_USED;
  sl.n = n;
  sl.K = K;
  sl.count = 1;
  sl.count_ub = 1;
  sl.seq = b->next_seq++;
  sl.F = 1.0;
  for (int q = 0; q < 64; ++q) sl.order[q] = (uint8_t)q;  // sorted by the natural key at first
  *slot = s;
  return SV_OK;
}

sv_status svb_remove(svb_state* b, int slot) {
  SVB_GUARD(b);
  if (slot < 0 || slot >= b->max_slots || b->slots[slot].state != SLOT_USED)
    return b_fail(b, SV_E_ARG, "svb_remove: slot not in use");
  b->slots[slot].state = SLOT_REMOVING;  // its terms are dropped by the next step
  return SV_OK;
}

sv_status svb_step(svb_state* b, const svb_gate* gates, int count) {
  SVB_GUARD(b);
  if (count < 0 || (count > 0 && !gates)) return b_fail(b, SV_E_ARG, "svb_step: bad gate list");
  // gate table: listed slots get their gate, other used slots the identity,
  // removed slots the drop marker
  std::vector<int> listed(b->max_slots, -1);
  for (int i = 0; i < count; ++i) {
    const svb_gate& g = gates[i];
    if (g.slot < 0 || g.slot >= b->max_slots || b->slots[g.slot].state != SLOT_USED)
      return b_fail(b, SV_E_ARG, "svb_step: slot not in use");
    if (listed[g.slot] >= 0) return b_fail(b, SV_E_ARG, "svb_step: two gates for one slot");
    if (g.m < 1 || g.m > 4 || !g.U) return b_fail(b, SV_E_ARG, "svb_step: bad m or U");
    uint64_t qm = 0;
    for (int t = 0; t < g.m; ++t) {
      if (g.qubits[t] < 0 || g.qubits[t] >= b->slots[g.slot].n || (qm >> g.qubits[t]) & 1ull)
        return b_fail(b, SV_E_ARG, "svb_step: bad qubit");
      qm |= 1ull << g.qubits[t];
    }
    if (!is_unitary(g.m, g.U)) return b_fail(b, SV_E_NOT_UNITARY, "svb_step: U is not unitary within 1e-10");
    listed[g.slot] = i;
  }
  const bool layer = b->layer_on;
  // the gate table: with one launch per step the two pinned table sets
  // alternate, and a set is rewritten once the step that read it is done
  const int par = layer ? b->tparity : 0;
  if (layer) {
    sv_status rc = b_cuda(b, cudaEventSynchronize(b->upload_ev[par]), "svb_step table reuse");
    if (rc != SV_OK) return rc;
    if (b->lev_pending[par]) {  // that step (two steps back) is done: its launch time is known
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, b->lev[par][0], b->lev[par][1]) == cudaSuccess)
        tune_record(b, b->lev_key[par], b->lev_shapes[par], b->lev_cfg[par], ms);
      cudaGetLastError();
      b->lev_pending[par] = false;
    }
  }
  SegGate* gh = b->gates_host + (size_t)par * b->max_slots;
  uint16_t* rh = b->rank_slot_host + (size_t)par * b->max_slots;
  int top = 0, maxn = 1, mmax = 0;
  uint64_t removed = 0, total = 0, cand = 0;
  bool may_truncate = false;
  for (int s = 0; s < b->max_slots; ++s) {
    const Slot& sl = b->slots[s];
    SegGate& gt = gh[s];
    const uint64_t cnt = layer ? sl.count_ub : sl.count;  // the host's exact count, or its bound
    if (sl.state == SLOT_FREE) {
      gt.m = -1;
      gt.K = 0;
      continue;
    }
    top = s + 1;
    total += cnt;
    if (sl.state == SLOT_REMOVING) {
      gt.m = -1;
      gt.K = 0;
      removed += cnt;
      continue;
    }
    const int gm = listed[s] >= 0 ? gates[listed[s]].m : 0;
    cand += cnt << gm;
    maxn = sl.n > maxn ? sl.n : maxn;
    std::memset(&gt, 0, sizeof(SegGate));
    gt.K = sl.K;
    // a slot can exceed its K after this step only if its count times the
    // gate's expansion does
    if ((cnt << gm) > sl.K) may_truncate = true;
    for (int q = 0; q < 64; ++q) gt.pos[q] = q < sl.n ? sl.order[q] : 64;
    if (listed[s] < 0) {  // identity: the slot keeps its order
      gt.m = 0;
      gt.re_nz[0] = 1;
      gt.U[0] = 1.0;
      continue;
    }
    const svb_gate& g = gates[listed[s]];
    gt.m = g.m;
    {  // the gate's sort order: its qubits at the bottom, the others in their present order
      int by_pos[64];
      for (int p = 0; p < 64; ++p) by_pos[p] = -1;
      for (int q = 0; q < sl.n; ++q) by_pos[sl.order[q]] = q;
      bool in_gate[64] = {};
      for (int t = 0; t < g.m; ++t) {
        in_gate[g.qubits[t]] = true;
        gt.pos[g.qubits[t]] = (uint8_t)t;
      }
      int next = g.m;
      for (int p = 0; p < 64; ++p) {
        const int q = by_pos[p];
        if (q >= 0 && !in_gate[q]) gt.pos[q] = (uint8_t)next++;
      }
    }
    mmax = g.m > mmax ? g.m : mmax;
    const int d = 1 << g.m;
    for (int t = 0; t < g.m; ++t) gt.q[t] = g.qubits[t];
    for (int ro = 0; ro < d; ++ro)
      for (int r = 0; r < d; ++r) {
        const double ur = g.U[2 * (ro * d + r)], ui = g.U[2 * (ro * d + r) + 1];
        gt.U[2 * (ro * d + r)] = ur;
        gt.U[2 * (ro * d + r) + 1] = ui;
        const bool rz = b->prec == SV_C128 ? ur != 0.0 : (float)ur != 0.0f;
        const bool iz = b->prec == SV_C128 ? ui != 0.0 : (float)ui != 0.0f;
        if (rz) gt.re_nz[ro] |= 1u << r;
        if (iz) gt.im_nz[ro] |= 1u << r;
      }
    for (int t = 0; t < g.m; ++t) gt.qs[t] = g.qubits[t];
    std::sort(gt.qs, gt.qs + g.m);
  }
  {  // segment ranks: the used slots in buffer order, which is their order of admission
    std::vector<std::pair<uint64_t, int>> used;
    for (int s = 0; s < top; ++s)
      if (b->slots[s].state == SLOT_USED) used.push_back({b->slots[s].seq, s});
    std::sort(used.begin(), used.end());
    for (size_t r = 0; r < used.size(); ++r) {
      gh[used[r].second].rank = (uint32_t)r;
      rh[r] = (uint16_t)used[r].second;
    }
  }
  ++b->steps;
  const uint64_t N = layer ? total : b->N;
  if (N == 0 || top == 0) {
    for (int s = 0; s < b->max_slots; ++s)
      if (b->slots[s].state == SLOT_REMOVING) b->slots[s] = Slot();
    if (!layer) b->N = 0;
    return SV_OK;
  }
  const uint64_t nkeep = N - removed;
  int segbits = 0;
  while ((1 << segbits) <= top) ++segbits;  // every real sort key is below the drop marker
  const int shift = maxn;
  const int nbits = shift + segbits;
  const uint64_t need = layer ? (cand > N ? cand : N) : (nkeep << mmax > N ? nkeep << mmax : N);
  sv_status rc = SV_OK;
  if (layer && b->pending && (need > b->cap || N > b->sort_cap || layer_grows(b, N, nkeep, mmax > 1 ? mmax : 1)))
    rc = b_settle(b);  // buffers in use by steps in flight are replaced only after those steps
  if (rc == SV_OK) rc = b_state_cap(b, need);
  if (rc == SV_OK) rc = b_sort_cap(b, N);
  if (rc != SV_OK) return rc;
  if (layer) {
    rc = step_layer(b, par, top, N, nkeep, shift, mmax);
    if (rc != SV_OK) return rc;
    for (int s = 0; s < b->max_slots; ++s) {
      Slot& sl = b->slots[s];
      if (sl.state == SLOT_REMOVING) {
        sl = Slot();  // its terms are dropped by the step just enqueued
        continue;
      }
      if (sl.state != SLOT_USED || s >= top) continue;
      for (int q = 0; q < sl.n; ++q) sl.order[q] = gh[s].pos[q];
      if (listed[s] >= 0) {  // the count after the gate's expansion and the top-k cut
        const uint64_t grown = sl.count_ub << gates[listed[s]].m;
        sl.count_ub = grown < sl.K ? grown : sl.K;
      }
    }
    b->tparity ^= 1;
    return SV_OK;
  }
  bool truncated = false;
  rc = step_kernels(b, top, N, nkeep, shift, nbits, mmax, may_truncate, truncated);
  if (rc != SV_OK) return rc;
  for (int s = 0; s < b->max_slots; ++s) {
    Slot& sl = b->slots[s];
    if (sl.state != SLOT_USED) continue;
    if (s < top)  // the segment is now sorted by this step's order
      for (int q = 0; q < sl.n; ++q) sl.order[q] = gh[s].pos[q];
    if (s < top) {
      const uint64_t* bh = b->bounds_host + (truncated ? 2 * b->max_slots : 0);  // the state's bounds
      const uint64_t a = bh[s], e = bh[b->max_slots + s];
      sl.offset = e > a ? a : 0;  // a slot with no terms keeps start all ones
      sl.count = e > a ? e - a : 0;
    }
    if (truncated && s < top) {
      const SegSel& st = b->sel_host[s];
      if (st.active && st.done == 1) {
        const double Sc = u128_to_double(st.cut_mass_hi, st.cut_mass_lo);
        const double SN = u128_to_double(st.total_mass_hi, st.total_mass_lo);
        sl.F = sl.F * (Sc / SN);
      }
    }
  }
  return SV_OK;
}

sv_status svb_set_autotune(svb_state* b, int on) {
  SVB_GUARD(b);
  b->autotune = on != 0;
  return SV_OK;
}

sv_status svb_set_layer_kernel(svb_state* b, int on) {
  SVB_GUARD(b);
  if ((on != 0) == b->layer_on) return SV_OK;
  for (const Slot& sl : b->slots)
    if (sl.state != SLOT_FREE) return b_fail(b, SV_E_STATE, "svb_set_layer_kernel: the batch must be empty");
  sv_status rc = b_settle(b);
  if (rc != SV_OK) return rc;
  if (on) {  // the device takes over the bookkeeping of the (empty) state
    b->lc_host->cur = (uint32_t)b->cur;
    b->lc_host->n_cur = b->N;
    rc = b_cuda(b, cudaMemcpyAsync(b->lc_dev, b->lc_host, sizeof(LayerCtl), cudaMemcpyHostToDevice, b->st),
                "svb_set_layer_kernel");
    if (rc == SV_OK) rc = b_cuda(b, cudaStreamSynchronize(b->st), "svb_set_layer_kernel");
    if (rc != SV_OK) return rc;
  }
  b->layer_on = on != 0;
  return SV_OK;
}

sv_status svb_layer_phase_times(svb_state* b, double* ms, int cap, int* count) {
  SVB_GUARD(b);
  if (!count || (cap > 0 && !ms)) return b_fail(b, SV_E_ARG, "svb_layer_phase_times: bad arguments");
  sv_status rc = b_settle(b);
  if (rc != SV_OK) return rc;
  *count = LP_COUNT;
  for (int i = 0; i < cap && i < LP_COUNT; ++i) ms[i] = 1e-6 * (double)b->lc_host->phase_ns[i];
  return SV_OK;
}

sv_status svb_set_graphs(svb_state* b, int on) {
  SVB_GUARD(b);
  b->graphs_on = on != 0;
  if (!b->graphs_on) drop_graphs(b);
  return SV_OK;
}

sv_status svb_graph_stats(const svb_state* b, uint64_t* captures, uint64_t* launches) {
  if (!b || !captures || !launches) return SV_E_ARG;
  *captures = b->graph_captures;
  *launches = b->graph_launches;
  return SV_OK;
}

sv_status svb_autotune_stats(const svb_state* b, uint64_t* trials, uint64_t* classes, uint64_t* settled) {
  if (!b || !trials || !classes || !settled) return SV_E_ARG;
  *trials = b->tune_trials;
  *classes = b->tune.size();
  uint64_t done = 0;
  for (const auto& kv : b->tune) {
    bool all = !kv.second.ms.empty();
    for (float t : kv.second.ms)
      if (t < 0.f) all = false;
    if (all) ++done;
  }
  *settled = done;
  return SV_OK;
}

sv_status svb_num_terms(svb_state* b, int slot, uint64_t* N) {
  SVB_GUARD(b);
  if (!N || slot < 0 || slot >= b->max_slots || b->slots[slot].state != SLOT_USED)
    return b_fail(b, SV_E_ARG, "svb_num_terms: slot not in use");
  {
    const sv_status rs = b_settle(b);  // after asynchronous steps: the slot's current range and mass
    if (rs != SV_OK) return rs;
  }
  *N = b->slots[slot].count;
  return SV_OK;
}

sv_status svb_retained_mass(svb_state* b, int slot, double* F) {
  SVB_GUARD(b);
  if (!F || slot < 0 || slot >= b->max_slots || b->slots[slot].state != SLOT_USED)
    return b_fail(b, SV_E_ARG, "svb_retained_mass: slot not in use");
  {
    const sv_status rs = b_settle(b);  // after asynchronous steps: the slot's current range and mass
    if (rs != SV_OK) return rs;
  }
  *F = b->slots[slot].F;
  return SV_OK;
}

sv_status svb_peak(svb_state* b, int slot, uint64_t* key, double* prob) {
  SVB_GUARD(b);
  if (!key || !prob || slot < 0 || slot >= b->max_slots || b->slots[slot].state != SLOT_USED)
    return b_fail(b, SV_E_ARG, "svb_peak: slot not in use");
  {
    const sv_status rs = b_settle(b);  // after asynchronous steps: the slot's current range and mass
    if (rs != SV_OK) return rs;
  }
  const Slot& sl = b->slots[slot];
  if (sl.count == 0) return b_fail(b, SV_E_STATE, "svb_peak: empty segment");
  // a truncation leaves no probabilities behind: recompute the segment's
  launch_amp_probs(b->prec, (const char*)b->amps[b->cur] + sl.offset * b->amp_bytes, sl.count,
                   b->probs[b->cur] + sl.offset, b->st);
  launch_peak(b->probs[b->cur] + sl.offset, b->keys[b->cur] + sl.offset, sl.count, b->ctl, b->st);
  sv_status rc = b_sync_ctl(b, "svb_peak");
  if (rc != SV_OK) return rc;
  *key = b->ctl_host->peak_z_lo;
  uint64_t bits = b->ctl_host->peak_z_hi;
  std::memcpy(prob, &bits, 8);
  return SV_OK;
}

sv_status svb_peak_async(svb_state* b, int slot, uint64_t* ticket) {
  SVB_GUARD(b);
  if (!ticket || slot < 0 || slot >= b->max_slots || b->slots[slot].state != SLOT_USED)
    return b_fail(b, SV_E_ARG, "svb_peak_async: slot not in use");
  const uint64_t t = b->next_ticket;
  const int r = (int)(t % PEAK_RING);
  if (b->ring_ticket[r]) return b_fail(b, SV_E_STATE, "svb_peak_async: too many readouts not yet collected");
  const Slot& sl = b->slots[slot];
  uint64_t* out = b->ring_dev + 4 * r;
  launch_seg_peak(b->keys, b->amps, b->prec, b->layer_on ? 1 : 0, b->lc_dev, b->bounds_dev, b->max_slots, b->F_dev,
                  slot, sl.offset, sl.count, b->cur, sl.F, b->peak_part, out, b->st);
  cudaMemcpyAsync(out + 3, &b->ctl->err, sizeof(uint32_t), cudaMemcpyDeviceToDevice, b->st);
  cudaMemcpyAsync(b->ring_host + 4 * r, out, sizeof(uint64_t) * 4, cudaMemcpyDeviceToHost, b->st);
  sv_status rc = b_cuda(b, cudaEventRecord(b->ring_ev[r], b->st), "svb_peak_async");
  if (rc != SV_OK) return rc;
  b->ring_ticket[r] = t + 1;
  b->next_ticket = t + 1;
  *ticket = t;
  return SV_OK;
}

sv_status svb_peak_wait(svb_state* b, uint64_t ticket, uint64_t* key, double* prob, double* F) {
  SVB_GUARD(b);
  const int r = (int)(ticket % PEAK_RING);
  if (!key || !prob || b->ring_ticket[r] != ticket + 1)
    return b_fail(b, SV_E_ARG, "svb_peak_wait: not a readout in flight");
  sv_status rc = b_cuda(b, cudaEventSynchronize(b->ring_ev[r]), "svb_peak_wait");
  if (rc != SV_OK) return rc;
  b->ring_ticket[r] = 0;
  const uint64_t* h = b->ring_host + 4 * r;
  const uint32_t err = (uint32_t)h[3];
  if (err) {
    b->broken = true;
    return b_fail(b, (err & ERR_TIMEOUT) ? SV_E_TIMEOUT : SV_E_STATE, "svb_peak_wait: device state error");
  }
  *key = h[0];
  std::memcpy(prob, &h[1], 8);
  if (F) std::memcpy(F, &h[2], 8);
  return SV_OK;
}

sv_status svb_export(svb_state* b, int slot, uint64_t* keys, double* amps, uint64_t cap, uint64_t* count) {
  SVB_GUARD(b);
  if (!count || slot < 0 || slot >= b->max_slots || b->slots[slot].state != SLOT_USED)
    return b_fail(b, SV_E_ARG, "svb_export: slot not in use");
  {
    const sv_status rs = b_settle(b);  // after asynchronous steps: the slot's current range and mass
    if (rs != SV_OK) return rs;
  }
  const Slot& sl = b->slots[slot];
  *count = sl.count;
  const uint64_t w = cap < sl.count ? cap : sl.count;
  if (w == 0) return SV_OK;
  sv_status rc = b_sort_cap(b, w);
  if (rc != SV_OK) return rc;
  double* tmp = (double*)b_alloc(b, w * 16);
  if (!tmp) return b_fail(b, SV_E_NOMEM, "svb_export: staging allocation failed");
  launch_amp_probs(b->prec, (const char*)b->amps[b->cur] + sl.offset * b->amp_bytes, w,
                   b->probs[b->cur] + sl.offset, b->st);
  launch_iota(b->sidx[0], w, b->st);
  launch_gather_terms(b->prec, b->sidx[0], w, b->keys[b->cur] + sl.offset,
                      (const char*)b->amps[b->cur] + sl.offset * b->amp_bytes, b->probs[b->cur] + sl.offset,
                      nullptr, tmp, nullptr, nullptr, b->st);
  if (keys) cudaMemcpyAsync(keys, b->keys[b->cur] + sl.offset, w * 8, cudaMemcpyDeviceToHost, b->st);
  if (amps) cudaMemcpyAsync(amps, tmp, w * 16, cudaMemcpyDeviceToHost, b->st);
  rc = b_cuda(b, cudaStreamSynchronize(b->st), "svb_export");
  b_free(b, tmp);
  return rc;
}

const char* svb_last_error(const svb_state* b) { return b ? b->err.c_str() : "null handle"; }

}  // extern "C"
