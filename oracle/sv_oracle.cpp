// CPU oracle for the sparse truncated state-vector method.
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
// call this file: only the tests, the smoke check and the CPU-baseline leg of
// the benchmark use it.  It shares no code with the CUDA library.
//
// It is a plain, single-threaded, deliberately slow restatement of what the
// paper's method computes:
//   * state: an ordered map basis-state key -> complex amplitude holding only
//     nonzero amplitudes, starting from the single term |0...0> (Sec. I and
//     Sec. II; keys are 64-bit integers, amplitudes complex128, Sec. V);
//   * gate: every group of basis states that differ only in the m target
//     bits is multiplied by the 2^m x 2^m unitary (Eq. 3 generalised,
//     Sec. IV-A); contributions to the same new basis state are summed; exact
//     zeros are not stored;
//   * truncation: terms ordered by decreasing probability, the p-mass cut
//     first, then the top-k cut, then renormalisation (Sec. III and
//     Sec. IV-B); the retained probability mass is multiplied into a running
//     product, the paper's fidelity estimate (Sec. III);
//   * readout: the most probable basis state (Sec. V).
//
// Readings where the paper is silent (each one is listed in the design
// notes):
//   R1 qubit i is bit i of the key; the local index of a gate on
//      qubits[0..m-1] is r = sum_t bit(key, qubits[t]) << t; U is row-major
//      U[r_out][r_in].
//   R2 amplitude arithmetic: for each output r_out the accumulator starts at
//      +0+0i and visits the present members in ascending r_in; each complex
//      multiply-accumulate is four fused multiply-adds in the fixed order
//      re = fma(ur, xr, re); re = fma(-ui, xi, re);
//      im = fma(ur, xi, im); im = fma(ui, xr, im).
//      In the complex64 form U is rounded to float and the same sequence
//      runs in float (fmaf).
//   R3 a term is dropped when re == 0 and im == 0 (no epsilon).
//   R4 prob = fma(re, re, im*im) in double (complex64 components are widened
//      to double first, which makes both products exact).
//   R5 canonical order: prob descending, then key ascending.
//   R6 masses are exact sums of floor(prob * 2^120) in 128-bit integers; a
//      mass is turned into a double by round-to-nearest-even.
//   R7 p-mass: T = fx(p * double(S_N)); c_p = the smallest c >= 1 whose
//      prefix mass S_c >= T; p >= 1 disables the p cut.
//   R8 c = min(c_p, K); if c == N nothing changes (no renormalisation);
//      otherwise the first c terms are kept and scaled by
//      s = 1 / sqrt(double(S_c)) (complex64: float(double(x) * s)), and the
//      retained product F *= double(S_c) / double(S_N).
//   R9 peak = first term in canonical order.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

namespace {

typedef unsigned __int128 u128;

struct Amp {
  double re, im;  // complex64 form: both hold float values exactly
};

struct Oracle {
  int n;
  uint64_t K;
  double p;
  int prec;  // 0 = complex128, 1 = complex64
  std::map<uint64_t, Amp> state;
  double F;
  // statistics of the last truncation
  uint64_t last_N, last_c;
  u128 last_SN, last_Sc;
};

// R4
double prob_of(const Amp& a) { return std::fma(a.re, a.re, a.im * a.im); }

// R6: floor(p * 2^120) for 0 <= p < 2^7, exactly.
u128 fx(double p) {
  if (!(p > 0.0)) return 0;
  int e = 0;
  double f = std::frexp(p, &e);                      // p = f * 2^e, f in [0.5, 1)
  uint64_t mant = (uint64_t)std::ldexp(f, 53);       // exact 53-bit integer
  int sh = e - 53 + 120;                             // p * 2^120 = mant * 2^sh
  if (sh >= 0) return ((u128)mant) << sh;
  if (sh <= -64) return 0;
  return (u128)(mant >> (-sh));
}

// R6: nearest double to S * 2^-120 (the integer conversion rounds to nearest
// even; the power-of-two scaling is exact).
double fx_to_double(u128 s) { return std::ldexp((double)s, -120); }

// R5
bool canon_less(uint64_t ka, double pa, uint64_t kb, double pb) {
  if (pa != pb) return pa > pb;
  return ka < kb;
}

struct Term {
  uint64_t key;
  double prob;
};

std::vector<Term> canonical_terms(const Oracle& o) {
  std::vector<Term> t;
  t.reserve(o.state.size());
  for (const auto& kv : o.state) t.push_back({kv.first, prob_of(kv.second)});
  std::sort(t.begin(), t.end(), [](const Term& a, const Term& b) {
    return canon_less(a.key, a.prob, b.key, b.prob);
  });
  return t;
}

}  // namespace

extern "C" {

void* or_create(int n, uint64_t K, double p, int prec) {
  if (n < 1 || n > 64 || K < 1 || !(p > 0.0) || (prec != 0 && prec != 1)) return nullptr;
  Oracle* o = new Oracle();
  o->n = n;
  o->K = K;
  o->p = p;
  o->prec = prec;
  o->F = 1.0;
  o->last_N = o->last_c = 0;
  o->last_SN = o->last_Sc = 0;
  o->state[0] = Amp{1.0, 0.0};  // |0...0>, a single term (Sec. I)
  return o;
}

void or_destroy(void* h) { delete (Oracle*)h; }

// Sec. IV-A / Eq. (3): apply a 2^m x 2^m unitary to the qubits q[0..m-1].
// U holds 2*4^m doubles, row-major U[r_out][r_in], interleaved (re, im).
int or_apply_gate(void* h, int m, const int* q, const double* U) {
  Oracle& o = *(Oracle*)h;
  if (m < 1 || m > 4) return -1;
  uint64_t Qmask = 0;
  for (int t = 0; t < m; t++) {
    if (q[t] < 0 || q[t] >= o.n) return -1;
    if (Qmask & (1ull << q[t])) return -1;
    Qmask |= 1ull << q[t];
  }
  const int d = 1 << m;

  // group the terms by the bits outside the gate (R1)
  std::map<uint64_t, size_t> group_of;
  std::vector<uint32_t> present;
  std::vector<Amp> x;
  for (const auto& kv : o.state) {
    uint64_t key = kv.first;
    uint64_t rest = key & ~Qmask;
    int r = 0;
    for (int t = 0; t < m; t++) r |= (int)((key >> q[t]) & 1ull) << t;
    auto it = group_of.find(rest);
    size_t g;
    if (it == group_of.end()) {
      g = present.size();
      group_of[rest] = g;
      present.push_back(0);
      x.resize(x.size() + d, Amp{0.0, 0.0});
    } else {
      g = it->second;
    }
    present[g] |= 1u << r;
    x[g * d + r] = kv.second;
  }

  std::map<uint64_t, Amp> out;
  for (const auto& gk : group_of) {
    uint64_t rest = gk.first;
    size_t g = gk.second;
    for (int ro = 0; ro < d; ro++) {
      Amp acc{0.0, 0.0};
      if (o.prec == 0) {
        double re = 0.0, im = 0.0;
        for (int ri = 0; ri < d; ri++) {
          if (!((present[g] >> ri) & 1u)) continue;
          double ur = U[2 * (ro * d + ri)], ui = U[2 * (ro * d + ri) + 1];
          const Amp& a = x[g * d + ri];
          re = std::fma(ur, a.re, re);
          re = std::fma(-ui, a.im, re);
          im = std::fma(ur, a.im, im);
          im = std::fma(ui, a.re, im);
        }
        acc = Amp{re, im};
      } else {
        float re = 0.0f, im = 0.0f;
        for (int ri = 0; ri < d; ri++) {
          if (!((present[g] >> ri) & 1u)) continue;
          float ur = (float)U[2 * (ro * d + ri)], ui = (float)U[2 * (ro * d + ri) + 1];
          const Amp& a = x[g * d + ri];
          float ar = (float)a.re, ai = (float)a.im;
          re = std::fmaf(ur, ar, re);
          re = std::fmaf(-ui, ai, re);
          im = std::fmaf(ur, ai, im);
          im = std::fmaf(ui, ar, im);
        }
        acc = Amp{(double)re, (double)im};
      }
      if (acc.re == 0.0 && acc.im == 0.0) continue;  // R3
      uint64_t key = rest;
      for (int t = 0; t < m; t++) key |= (uint64_t)((ro >> t) & 1) << q[t];
      out[key] = acc;
    }
  }
  o.state.swap(out);
  return 0;
}

// Sec. III / Sec. IV-B: p-mass cut, then top-k cut, then renormalisation.
int or_truncate(void* h, uint64_t* kept, double* retained_fraction) {
  Oracle& o = *(Oracle*)h;
  std::vector<Term> t = canonical_terms(o);
  const uint64_t N = t.size();
  u128 SN = 0;
  for (const Term& x : t) SN += fx(x.prob);
  uint64_t cp = N;
  if (o.p < 1.0 && N > 0) {
    u128 T = fx(o.p * fx_to_double(SN));
    u128 S = 0;
    for (uint64_t c = 1; c <= N; c++) {
      S += fx(t[c - 1].prob);
      if (S >= T) {
        cp = c;
        break;
      }
    }
  }
  uint64_t c = std::min<uint64_t>(cp, o.K);
  o.last_N = N;
  o.last_SN = SN;
  double f = 1.0;
  if (c < N) {
    u128 Sc = 0;
    for (uint64_t i = 0; i < c; i++) Sc += fx(t[i].prob);
    double s = 1.0 / std::sqrt(fx_to_double(Sc));
    std::map<uint64_t, Amp> out;
    for (uint64_t i = 0; i < c; i++) {
      Amp a = o.state[t[i].key];
      if (o.prec == 0) {
        a.re = a.re * s;
        a.im = a.im * s;
      } else {
        a.re = (double)(float)(a.re * s);
        a.im = (double)(float)(a.im * s);
      }
      out[t[i].key] = a;
    }
    o.state.swap(out);
    f = fx_to_double(Sc) / fx_to_double(SN);
    o.F = o.F * f;
    o.last_c = c;
    o.last_Sc = Sc;
  } else {
    o.last_c = N;
    o.last_Sc = SN;
  }
  if (kept) *kept = o.state.size();
  if (retained_fraction) *retained_fraction = f;
  return 0;
}

// Sec. V: the most probable basis state.
int or_peak(void* h, uint64_t* key, double* prob) {
  Oracle& o = *(Oracle*)h;
  if (o.state.empty()) return -6;
  bool first = true;
  uint64_t bk = 0;
  double bp = 0.0;
  for (const auto& kv : o.state) {
    double pr = prob_of(kv.second);
    if (first || canon_less(kv.first, pr, bk, bp)) {
      bk = kv.first;
      bp = pr;
      first = false;
    }
  }
  *key = bk;
  *prob = bp;
  return 0;
}

uint64_t or_num_terms(void* h) { return ((Oracle*)h)->state.size(); }

double or_retained_mass(void* h) { return ((Oracle*)h)->F; }

// Terms in canonical order: keys[i], amps[2i], amps[2i+1], probs[i]
// (probs may be null).  Writes min(cap, N) entries; *count = N.
int or_export(void* h, uint64_t* keys, double* amps, double* probs, uint64_t cap,
              uint64_t* count) {
  Oracle& o = *(Oracle*)h;
  std::vector<Term> t = canonical_terms(o);
  uint64_t w = std::min<uint64_t>(cap, t.size());
  for (uint64_t i = 0; i < w; i++) {
    const Amp& a = o.state[t[i].key];
    if (keys) keys[i] = t[i].key;
    if (amps) {
      amps[2 * i] = a.re;
      amps[2 * i + 1] = a.im;
    }
    if (probs) probs[i] = t[i].prob;
  }
  *count = t.size();
  return 0;
}

// Replace the state (checkpoint / test hook).  Zero amplitudes are not
// stored; duplicate keys or keys outside n bits are rejected.  In the
// complex64 form the components are rounded to float.
int or_load(void* h, const uint64_t* keys, const double* amps, uint64_t N) {
  Oracle& o = *(Oracle*)h;
  std::map<uint64_t, Amp> s;
  for (uint64_t i = 0; i < N; i++) {
    if (o.n < 64 && (keys[i] >> o.n) != 0) return -1;
    if (s.count(keys[i])) return -1;
    Amp a{amps[2 * i], amps[2 * i + 1]};
    if (o.prec == 1) {
      a.re = (double)(float)a.re;
      a.im = (double)(float)a.im;
    }
    if (a.re == 0.0 && a.im == 0.0) continue;
    s[keys[i]] = a;
  }
  o.state.swap(s);
  return 0;
}

// Exact total mass as a 128-bit fixed-point number (hi, lo words).
void or_total_mass_fx(void* h, uint64_t* hi, uint64_t* lo) {
  Oracle& o = *(Oracle*)h;
  u128 S = 0;
  for (const auto& kv : o.state) S += fx(prob_of(kv.second));
  *hi = (uint64_t)(S >> 64);
  *lo = (uint64_t)S;
}

// Statistics of the last truncation: N before, c kept, S_N and S_c.
void or_last_cut(void* h, uint64_t* N, uint64_t* c, uint64_t* sn_hi, uint64_t* sn_lo,
                 uint64_t* sc_hi, uint64_t* sc_lo) {
  Oracle& o = *(Oracle*)h;
  *N = o.last_N;
  *c = o.last_c;
  *sn_hi = (uint64_t)(o.last_SN >> 64);
  *sn_lo = (uint64_t)o.last_SN;
  *sc_hi = (uint64_t)(o.last_Sc >> 64);
  *sc_lo = (uint64_t)o.last_Sc;
}

// Building blocks exposed for pinning tests.
void or_fx(double p, uint64_t* hi, uint64_t* lo) {
  u128 v = fx(p);
  *hi = (uint64_t)(v >> 64);
  *lo = (uint64_t)v;
}

double or_fx_to_double(uint64_t hi, uint64_t lo) {
  return fx_to_double(((u128)hi << 64) | lo);
}

double or_prob(double re, double im) { return prob_of(Amp{re, im}); }

}  // extern "C"
