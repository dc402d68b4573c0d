// Host-side helpers shared by the single-state and batched C ABI files.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include "internal.h"

namespace sv {

// Sort-key permutation of a gate: gate qubit q[t] at bit t, the other
// qubits above in the order of order[] (order[b] = bit of qubit b in the
// sort key the state is currently sorted by).  Writes the forward and
// inverse nibble tables, and the new order into next[] (may alias order).
inline void build_perm(int n, int m, const int* q, const int* order, BitPerm* bp, int* next) {
  int pos[64];
  for (int b = 0; b < 64; ++b) pos[b] = -1;
  for (int t = 0; t < m; ++t) pos[q[t]] = t;
  int by_bit[64];
  for (int b = 0; b < 64; ++b) by_bit[b] = -1;
  for (int b = 0; b < n; ++b) by_bit[order[b]] = b;
  int nextbit = m;
  for (int p = 0; p < n; ++p) {
    const int b = by_bit[p];
    if (b >= 0 && pos[b] < 0) pos[b] = nextbit++;
  }
  std::memset(bp, 0, sizeof(BitPerm));
  for (int k = 0; k < 16; ++k)
    for (int v = 0; v < 16; ++v)
      for (int j = 0; j < 4; ++j)
        if ((v >> j) & 1) {
          const int b = 4 * k + j;
          if (b < n) bp->fwd[k][v] |= 1ull << pos[b];
        }
  int from[64];
  for (int b = 0; b < 64; ++b) from[b] = -1;
  for (int b = 0; b < n; ++b) from[pos[b]] = b;
  for (int k = 0; k < 16; ++k)
    for (int v = 0; v < 16; ++v)
      for (int j = 0; j < 4; ++j)
        if ((v >> j) & 1) {
          const int p = 4 * k + j;
          if (p < n) bp->inv[k][v] |= 1ull << from[p];
        }
  for (int b = 0; b < n; ++b) next[b] = pos[b];
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
inline double u128_to_double(uint64_t hi, uint64_t lo) {
  unsigned __int128 v = ((unsigned __int128)hi << 64) | lo;
  return std::ldexp((double)v, -120);
}

}  // namespace sv
