// mg_internal.h -- declarations shared by the engine's own translation units.
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/mg.h"

namespace mg {

constexpr int kMaxGluons = 5;      // g g -> t tbar g g g
constexpr int kMaxNcol = 120;      // 5!
constexpr int kMaxSeq = 105;       // canonical gluon sequences of length 1..K-1 for K = 5
constexpr int kPage = 32;          // AoSoA page: events per page

// Count one kernel launch of this library (process-wide, thread-safe; read by mg_kernel_launches).
void note_launch();

inline int gluons_of(mg_process p) { return static_cast<int>(p) + 2; }
inline int npar_of(mg_process p) { return static_cast<int>(p) + 4; }
inline int factorial(int n) { int f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

// ----------------------------------------------------------------------------------------
// Exact colour matrix of one quark line + K gluons (mg_colour.cpp):
// C(sigma,tau) = Tr(T^sigma (T^tau)^dagger) = num / den.
// ----------------------------------------------------------------------------------------
void colour_matrix_exact(int K, std::vector<int64_t>& num, int64_t& den);

// ----------------------------------------------------------------------------------------
// Recursion tables for K gluons (mg_tables.cpp).  A "slot reference" packs a canonical gluon
// sequence slot and a sign: ref = (slot << 1) | negative.  Canonical sequences of length >= 2
// have seq[0] < seq[L-1]; the reversed sequence carries the sign (-1)^(L+1) (reflection
// identity of colour-ordered gluon currents).
// ----------------------------------------------------------------------------------------
struct Tables {
  int K, ncol, nseq;
  // canonical sequences: length, subset mask; splits into (L,R) and (A,B,C) as slot refs
  uint8_t seq_len[kMaxSeq];
  uint8_t seq_mask[kMaxSeq];
  int16_t seq_v3[kMaxSeq][kMaxGluons - 1][2];
  int16_t seq_v4[kMaxSeq][6][3];
  uint8_t seq_nv3[kMaxSeq], seq_nv4[kMaxSeq];
  // permutations sigma in lexicographic order (= jamp index)
  uint8_t perm[kMaxNcol][kMaxGluons];
  uint8_t lcp[kMaxNcol];                        // common prefix length with the previous sigma
  uint8_t prefix_mask[kMaxNcol][kMaxGluons];    // mask of sigma[0..m) for m = 0..K-1
  // sub[c][j][m] = slot ref of sigma[j..m), 0 <= j < m <= K, (j, m) != (0, K)
  int16_t sub[kMaxNcol][kMaxGluons][kMaxGluons + 1];
  // full-length sigma: canonical flag, index into the full-current table, its splits
  int16_t full_idx[kMaxNcol];                   // >= 0: canonical, own index; < 0: -(idx of reverse)-1
  int nfull;
  int16_t full_v3[kMaxNcol / 2][kMaxGluons - 1][2];
  int16_t full_v4[kMaxNcol / 2][6][3];
  uint8_t full_nv3[kMaxNcol / 2], full_nv4[kMaxNcol / 2];
  uint8_t full_split_mask[kMaxNcol / 2][kMaxGluons - 1];   // mask of the left part of each V3 split
  // currents shared between gluon-helicity combinations: canonical sequence s with the helicities of its
  // own gluons h (2^len(s) of them) is item share_base[s] + h; share_n items per event
  int16_t share_base[kMaxSeq];
  int share_n;
  // quark-line prefixes shared the same way: the row spinor after the first m gluons of a colour ordering
  // (m = 1 .. pref_levels), for every helicity assignment of those gluons and both top helicities.
  // Level m's node (p, h, a) -- p = ordering / (K - m)!, h = the prefix gluons' helicities in ordering
  // order (bit j: gluon perm[.][j]), a = top helicity -- is item pref_off[m] + ((p << m | h) << 1 | a)
  // (8 doubles) after the share_n current items (24 doubles each); share_stride doubles per event,
  // interleaved by page of 32 events like the per-event record (double d of event e at
  // (e / 32) * share_stride * 32 + d * 32 + e % 32).
  int pref_levels;
  int pref_off[kMaxGluons];
  int share_stride;
};

// helicity bits of the gluons in mask, packed (bit g of gc -> the rank of g among mask's bits), and back
inline constexpr int pext_bits(int gc, int mask) {
  int r = 0, k = 0;
  for (int g = 0; g < kMaxGluons; ++g)
    if ((mask >> g) & 1) r |= ((gc >> g) & 1) << k++;
  return r;
}
inline constexpr int pdep_bits(int h, int mask) {
  int r = 0, k = 0;
  for (int g = 0; g < kMaxGluons; ++g)
    if ((mask >> g) & 1) r |= ((h >> k++) & 1) << g;
  return r;
}

void build_tables(int K, Tables& t);

}  // namespace mg
