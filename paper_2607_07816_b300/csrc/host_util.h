// Host-side helpers shared by the single-state and batched C ABI files.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include "internal.h"

namespace sv {

// Tables of a gate on stored keys (see BitPerm): order[b] is the bit of
// qubit b in the stored keys before the gate.  Writes the sort-key
// permutation (fwd: stored -> sort key; inv: identity), the natural-key table
// of the outputs, the gate qubits' stored positions qpos[t], and the qubit
// order after the gate into next[] (may alias order).
inline void build_gate_tables(int n, int m, const int* q, const int* order, GateTables* t, int* qpos, int* next) {
  int pos[64];  // qubit -> bit after the gate
  for (int b = 0; b < 64; ++b) pos[b] = -1;
  for (int k = 0; k < m; ++k) pos[q[k]] = k;
  int by_bit[64];  // stored bit -> qubit, before the gate
  for (int b = 0; b < 64; ++b) by_bit[b] = -1;
  for (int b = 0; b < n; ++b) by_bit[order[b]] = b;
  int nextbit = m;
  for (int p = 0; p < n; ++p) {
    const int b = by_bit[p];
    if (b >= 0 && pos[b] < 0) pos[b] = nextbit++;
  }
  std::memset(&t->perm, 0, sizeof(BitPerm));
  std::memset(t->nat, 0, sizeof(t->nat));
  for (int k = 0; k < 16; ++k)
    for (int v = 0; v < 16; ++v)
      for (int j = 0; j < 4; ++j)
        if ((v >> j) & 1) {
          const int p = 4 * k + j;
          if (p >= n) continue;
          t->perm.fwd[k][v] |= 1ull << pos[by_bit[p]];  // old stored bit p holds qubit by_bit[p]
          t->perm.inv[k][v] |= 1ull << p;
        }
  int qubit_at[64];  // bit after the gate -> qubit
  for (int b = 0; b < n; ++b) qubit_at[pos[b]] = b;
  for (int k = 0; k < 16; ++k)
    for (int v = 0; v < 16; ++v)
      for (int j = 0; j < 4; ++j)
        if ((v >> j) & 1) {
          const int p = 4 * k + j;
          if (p < n) t->nat[k][v] |= 1ull << qubit_at[p];
        }
  for (int k = 0; k < m; ++k) qpos[k] = order[q[k]];
  for (int b = 0; b < n; ++b) next[b] = pos[b];
}

// The natural-key table of stored keys in the qubit order `order`.
inline void build_nat_table(int n, const int* order, uint64_t (*nat)[16]) {
  int qubit_at[64];
  for (int b = 0; b < n; ++b) qubit_at[order[b]] = b;
  std::memset(nat, 0, sizeof(uint64_t) * 256);
  for (int k = 0; k < 16; ++k)
    for (int v = 0; v < 16; ++v)
      for (int j = 0; j < 4; ++j)
        if ((v >> j) & 1) {
          const int p = 4 * k + j;
          if (p < n) nat[k][v] |= 1ull << qubit_at[p];
        }
}

inline bool is_unitary(int m, const double* U) {
  const int d = 1 << m;
  for (int i = 0; i < 2 * d * d; ++i)
    if (!std::isfinite(U[i])) return false;
  double worst = 0.0;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double re = 0.0, im = 0.0;  // (U^dagger U)[a][b] = sum_r conj(U[r][a]) U[r][b]
      for (int r = 0; r < d; ++r) {
        double ar = U[2 * (r * d + a)], ai = U[2 * (r * d + a) + 1];
        double br = U[2 * (r * d + b)], bi = U[2 * (r * d + b) + 1];
        re += ar * br + ai * bi;
        im += ar * bi - ai * br;
      }
      if (a == b) re -= 1.0;
      double v = std::fabs(re) > std::fabs(im) ? std::fabs(re) : std::fabs(im);
      worst = v > worst ? v : worst;
    }
  return worst <= 1e-10;
}

// Nearest double to a 128-bit fixed-point mass (LSB 2^-120).
// floor(v * 2^120) of a non-negative double, exactly: the fixed point of the
// probability masses (the device kernels convert probabilities the same
// way).  Zero for subnormal or negative input; values of 128 and above do
// not fit and saturate.
inline unsigned __int128 fx_from_double(double v) {
  uint64_t b;
  std::memcpy(&b, &v, sizeof(b));
  const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
  if (e == 0 || (b >> 63)) return 0;
  const uint64_t mant = (b & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = (int)e - 955;  // v * 2^120 = mant * 2^(e - 1075 + 120)
  if (sh >= 0) return sh > 74 ? ~(unsigned __int128)0 : ((unsigned __int128)mant) << sh;
  if (sh <= -64) return 0;
  return (unsigned __int128)(mant >> (-sh));
}

inline double u128_to_double(uint64_t hi, uint64_t lo) {
  unsigned __int128 v = ((unsigned __int128)hi << 64) | lo;
  return std::ldexp((double)v, -120);
}

}  // namespace sv
