// mg_colour.cpp -- exact colour matrix for one quark line and K gluons.
//
// Colour decomposition (Mangano-Parke, Phys. Rep. 200 (1991) 301): with one quark line,
// M = sum_sigma (T^{a_sigma1} ... T^{a_sigmaK})_{i j} A(sigma), so the colour sum of |M|^2 is the
// quadratic form A^dagger C A with C(sigma,tau) = Tr(T^{sigma1}..T^{sigmaK} T^{tauK}..T^{tau1}).
//
// Method: every SU(N) gluon is a U(N) gluon minus its U(1) part,
//   sum_a (T^a)_{ij} (T^a)_{kl} = 1/2 delta_il delta_kj - 1/(2N) delta_ij delta_kl.
// Expanding the product over the K gluons, each subset S of gluons taking the U(1) term, a U(N)
// contraction only permutes index lines, so every term is N^(number of closed index loops):
//   C(sigma,tau) 2^K N^K = sum_S (-1)^|S| N^(K - |S| + loops(S)),
// an integer evaluated here exactly with a union-find over the 2K index lines of the trace.
// (The CPU reference computes the same matrix by recursive Fierz reduction instead.)
#include <algorithm>
#include <numeric>
#include <vector>

#include "mg_internal.h"

namespace mg {

namespace {

struct UnionFind {
  int p[2 * kMaxGluons];
  explicit UnionFind(int n) { for (int i = 0; i < n; ++i) p[i] = i; }
  int find(int x) { while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; } return x; }
  void join(int a, int b) { a = find(a); b = find(b); if (a != b) p[a] = b; }
};

int64_t ipow(int64_t b, int e) { int64_t r = 1; while (e-- > 0) r *= b; return r; }

// C(sigma,tau) * 2^K N^K for N = 3
int64_t scaled_entry(int K, const int* sigma, const int* tau) {
  const int N = 3;
  int n = 2 * K;
  int word[2 * kMaxGluons];
  for (int i = 0; i < K; ++i) { word[i] = sigma[i]; word[K + i] = tau[K - 1 - i]; }
  int pos[kMaxGluons][2];
  int seen[kMaxGluons] = {0};
  for (int p = 0; p < n; ++p) pos[word[p]][seen[word[p]]++] = p;
  int64_t total = 0;
  for (int S = 0; S < (1 << K); ++S) {
    // index line i_p enters generator p; i_{p+1} leaves it (cyclic)
    UnionFind uf(n);
    for (int g = 0; g < K; ++g) {
      int p = pos[g][0], q = pos[g][1];
      int p1 = (p + 1) % n, q1 = (q + 1) % n;
      if ((S >> g) & 1) { uf.join(p, p1); uf.join(q, q1); }   // U(1) part: generator -> identity
      else { uf.join(p, q1); uf.join(q, p1); }               // U(N) exchange
    }
    int loops = 0;
    for (int i = 0; i < n; ++i) if (uf.find(i) == i) ++loops;
    int s = __builtin_popcount(S);
    int64_t term = ipow(N, K - s + loops);
    total += (s & 1) ? -term : term;
  }
  return total;
}

}  // namespace

void colour_matrix_exact(int K, std::vector<int64_t>& num, int64_t& den) {
  std::vector<int> base(K);
  std::iota(base.begin(), base.end(), 0);
  std::vector<std::vector<int>> perms;
  do { perms.push_back(base); } while (std::next_permutation(base.begin(), base.end()));
  int ncol = static_cast<int>(perms.size());
  num.assign(static_cast<size_t>(ncol) * ncol, 0);
  den = ipow(2, K) * ipow(3, K);
  for (int s = 0; s < ncol; ++s)
    for (int t = 0; t < ncol; ++t) num[static_cast<size_t>(s) * ncol + t] = scaled_entry(K, perms[s].data(), perms[t].data());
  int64_t g = den;
  for (int64_t v : num) g = std::gcd(g, v < 0 ? -v : v);
  if (g > 1) {
    for (auto& v : num) v /= g;
    den /= g;
  }
}

}  // namespace mg
