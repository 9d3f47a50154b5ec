// mg_tables.cpp -- index tables of the colour-ordered Berends-Giele recursion (host side).
//
// The per-event work of Sec. 2 of the paper (every Feynman diagram into colour-flow amplitudes)
// is organised here as the colour-ordered recursion of Berends and Giele (Nucl. Phys. B306
// (1988) 759): an off-shell gluon current J(seq) for every ordered gluon sequence, built from
// its splits into two (three-gluon vertex) and three (four-gluon vertex) consecutive parts, and
// quark-line currents for every prefix of a colour ordering.  Every tree diagram is summed
// exactly once per colour ordering.  Two identities cut the work:
//   * reflection: J(reversed seq) = (-1)^(L+1) J(seq), so only sequences with seq[0] < seq[L-1]
//     are computed ("canonical");
//   * prefixes of consecutive orderings in lexicographic order are shared (a depth-first walk
//     recomputes only the prefixes after the common part).
#include <algorithm>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "mg_internal.h"

namespace mg {

namespace {

int16_t pack(int slot, bool neg) { return static_cast<int16_t>((slot << 1) | (neg ? 1 : 0)); }

}  // namespace

void build_tables(int K, Tables& t) {
  std::memset(&t, 0, sizeof(t));
  t.K = K;
  // canonical sequences of length 1..K-1
  std::map<std::vector<int>, int> slot_of;
  std::vector<std::vector<int>> seqs;
  for (int g = 0; g < K; ++g) { slot_of[{g}] = static_cast<int>(seqs.size()); seqs.push_back({g}); }
  for (int L = 2; L <= K - 1; ++L) {
    // all ordered sequences of L distinct gluons, lexicographic
    std::vector<int> idx(K);
    std::iota(idx.begin(), idx.end(), 0);
    std::vector<std::vector<int>> all;
    std::vector<int> cur;
    std::vector<bool> used(K, false);
    // depth-first enumeration
    std::vector<int> stack;
    auto rec = [&](auto&& self) -> void {
      if (static_cast<int>(cur.size()) == L) { all.push_back(cur); return; }
      for (int g = 0; g < K; ++g) {
        if (used[g]) continue;
        used[g] = true; cur.push_back(g);
        self(self);
        cur.pop_back(); used[g] = false;
      }
    };
    rec(rec);
    for (auto& s : all)
      if (s.front() < s.back()) { slot_of[s] = static_cast<int>(seqs.size()); seqs.push_back(s); }
  }
  t.nseq = static_cast<int>(seqs.size());
  t.share_n = 0;
  for (int i = 0; i < t.nseq; ++i) {
    t.share_base[i] = static_cast<int16_t>(t.share_n);
    t.share_n += 1 << seqs[i].size();
  }
  t.pref_levels = K - 1 < 3 ? K - 1 : 3;
  int nodes = 0;
  for (int m = 0; m < kMaxGluons; ++m) t.pref_off[m] = 0;
  for (int m = 1; m <= t.pref_levels; ++m) {
    int orderings = 1;   // ordered prefixes of m gluons: K! / (K - m)!
    for (int i = 0; i < m; ++i) orderings *= K - i;
    t.pref_off[m] = nodes;
    nodes += (orderings << m) * 2;
  }
  t.share_stride = t.share_n * 24 + nodes * 8;
  auto ref = [&](const std::vector<int>& s) -> int16_t {
    if (s.size() == 1) return pack(s[0], false);
    if (s.front() < s.back()) return pack(slot_of.at(s), false);
    std::vector<int> r(s.rbegin(), s.rend());
    bool neg = (s.size() % 2) == 0;   // (-1)^(L+1)
    return pack(slot_of.at(r), neg);
  };
  auto mask_of = [](const std::vector<int>& s) { int m = 0; for (int g : s) m |= 1 << g; return m; };
  auto sub = [](const std::vector<int>& s, int a, int b) { return std::vector<int>(s.begin() + a, s.begin() + b); };
  for (int i = 0; i < t.nseq; ++i) {
    const auto& s = seqs[i];
    int L = static_cast<int>(s.size());
    t.seq_len[i] = static_cast<uint8_t>(L);
    t.seq_mask[i] = static_cast<uint8_t>(mask_of(s));
    int n3 = 0, n4 = 0;
    for (int a = 1; a < L; ++a) {
      t.seq_v3[i][n3][0] = ref(sub(s, 0, a));
      t.seq_v3[i][n3][1] = ref(sub(s, a, L));
      ++n3;
    }
    for (int a = 1; a < L; ++a)
      for (int b = a + 1; b < L; ++b) {
        t.seq_v4[i][n4][0] = ref(sub(s, 0, a));
        t.seq_v4[i][n4][1] = ref(sub(s, a, b));
        t.seq_v4[i][n4][2] = ref(sub(s, b, L));
        ++n4;
      }
    t.seq_nv3[i] = static_cast<uint8_t>(n3);
    t.seq_nv4[i] = static_cast<uint8_t>(n4);
  }
  // colour orderings
  std::vector<int> p(K);
  std::iota(p.begin(), p.end(), 0);
  std::vector<std::vector<int>> perms;
  do { perms.push_back(p); } while (std::next_permutation(p.begin(), p.end()));
  t.ncol = static_cast<int>(perms.size());
  std::map<std::vector<int>, int> full_of;
  t.nfull = 0;
  for (int c = 0; c < t.ncol; ++c) {
    const auto& s = perms[c];
    for (int g = 0; g < K; ++g) t.perm[c][g] = static_cast<uint8_t>(s[g]);
    int l = 0;
    if (c > 0)
      while (l < K && perms[c - 1][l] == s[l]) ++l;
    t.lcp[c] = static_cast<uint8_t>(l);
    for (int m = 0; m < K; ++m) t.prefix_mask[c][m] = static_cast<uint8_t>(mask_of(sub(s, 0, m)));
    for (int j = 0; j < K; ++j)
      for (int m = j + 1; m <= K; ++m)
        if (!(j == 0 && m == K)) t.sub[c][j][m] = ref(sub(s, j, m));
    if (s.front() < s.back()) {
      int f = t.nfull++;
      full_of[s] = f;
      t.full_idx[c] = static_cast<int16_t>(f);
      int n3 = 0, n4 = 0;
      for (int a = 1; a < K; ++a) {
        t.full_v3[f][n3][0] = ref(sub(s, 0, a));
        t.full_v3[f][n3][1] = ref(sub(s, a, K));
        t.full_split_mask[f][n3] = static_cast<uint8_t>(mask_of(sub(s, 0, a)));
        ++n3;
      }
      for (int a = 1; a < K; ++a)
        for (int b = a + 1; b < K; ++b) {
          t.full_v4[f][n4][0] = ref(sub(s, 0, a));
          t.full_v4[f][n4][1] = ref(sub(s, a, b));
          t.full_v4[f][n4][2] = ref(sub(s, b, K));
          ++n4;
        }
      t.full_nv3[f] = static_cast<uint8_t>(n3);
      t.full_nv4[f] = static_cast<uint8_t>(n4);
    }
  }
  for (int c = 0; c < t.ncol; ++c) {
    const auto& s = perms[c];
    if (!(s.front() < s.back())) {
      std::vector<int> r(s.rbegin(), s.rend());
      t.full_idx[c] = static_cast<int16_t>(-full_of.at(r) - 1);
    }
  }
}

}  // namespace mg
