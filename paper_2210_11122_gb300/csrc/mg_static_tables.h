// mg_static_tables.h -- the Berends-Giele recursion tables of mg_tables.cpp, built at compile time.
//
// Same content and numbering as the run-time tables (canonical gluon sequences: the K single gluons,
// then the sequences of length 2, 3, ... K-1 with seq[0] < seq[L-1] in lexicographic order; colour
// orderings sigma = permutations of the K gluons in lexicographic order = jamp index), as constexpr
// data, so that a kernel can expand the whole recursion into straight-line code: every current index,
// every sign of the reflection identity J(reversed) = (-1)^(L+1) J(seq) and every subset mask becomes
// a constant, and the per-thread current arrays stay in registers instead of local memory.
#pragma once

namespace mg {
namespace st {

constexpr int kSeqMax = 105;   // canonical sequences for K = 5
constexpr int kColMax = 120;   // 5!
constexpr int kFullMax = 60;   // canonical full-length orderings for K = 5

struct Tab {
  int K = 0, nseq = 0, ncol = 0, nfull = 0;
  int len[kSeqMax] = {};
  int mask[kSeqMax] = {};
  int el[kSeqMax][5] = {};
  int nv3[kSeqMax] = {};
  int nv4[kSeqMax] = {};
  int v3[kSeqMax][4][2] = {};    // splits into two consecutive parts: slot refs (slot << 1 | negative)
  int v4[kSeqMax][6][3] = {};    // splits into three consecutive parts
  int perm[kColMax][5] = {};
  int lcp[kColMax] = {};         // common prefix length with the previous ordering
  int pmask[kColMax][5] = {};    // subset mask of sigma[0..m)
  int sub[kColMax][5][6] = {};   // slot ref of sigma[j..m), (j, m) != (0, K)
  int fidx[kColMax] = {};        // >= 0: canonical full ordering, own index; < 0: -(index of reverse) - 1
  int fnv3[kFullMax] = {};
  int fnv4[kFullMax] = {};
  int fv3[kFullMax][4][2] = {};
  int fv4[kFullMax][6][3] = {};
};

constexpr int find_seq(const Tab& t, const int* s, int n) {
  for (int i = 0; i < t.nseq; ++i) {
    if (t.len[i] != n) continue;
    bool eq = true;
    for (int k = 0; k < n; ++k)
      if (t.el[i][k] != s[k]) eq = false;
    if (eq) return i;
  }
  return -1;
}

// slot reference of the consecutive part s[a..b)
constexpr int ref_of(const Tab& t, const int* s, int a, int b) {
  const int n = b - a;
  if (n == 1) return s[a] << 1;
  int f[5] = {};
  if (s[a] < s[b - 1]) {
    for (int k = 0; k < n; ++k) f[k] = s[a + k];
    return find_seq(t, f, n) << 1;
  }
  for (int k = 0; k < n; ++k) f[k] = s[b - 1 - k];
  return (find_seq(t, f, n) << 1) | (n % 2 == 0 ? 1 : 0);
}

constexpr int mask_of(const int* s, int a, int b) {
  int m = 0;
  for (int k = a; k < b; ++k) m |= 1 << s[k];
  return m;
}

// the ordered tuples of L distinct gluons out of K, lexicographic: code = sum s[i] K^(L-1-i)
constexpr bool tuple_of(int K, int L, int code, int* s) {
  for (int i = L - 1; i >= 0; --i) {
    s[i] = code % K;
    code /= K;
  }
  for (int i = 0; i < L; ++i)
    for (int j = i + 1; j < L; ++j)
      if (s[i] == s[j]) return false;
  return true;
}

constexpr int ipow(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

constexpr Tab make_tab(int K) {
  Tab t{};
  t.K = K;
  for (int g = 0; g < K; ++g) {
    t.len[g] = 1;
    t.el[g][0] = g;
    t.mask[g] = 1 << g;
  }
  t.nseq = K;
  for (int L = 2; L <= K - 1; ++L)
    for (int code = 0; code < ipow(K, L); ++code) {
      int s[5] = {};
      if (!tuple_of(K, L, code, s) || !(s[0] < s[L - 1])) continue;
      const int i = t.nseq++;
      t.len[i] = L;
      for (int k = 0; k < L; ++k) t.el[i][k] = s[k];
      t.mask[i] = mask_of(s, 0, L);
    }
  for (int i = K; i < t.nseq; ++i) {
    const int L = t.len[i];
    const int* s = t.el[i];
    int n3 = 0, n4 = 0;
    for (int a = 1; a < L; ++a) {
      t.v3[i][n3][0] = ref_of(t, s, 0, a);
      t.v3[i][n3][1] = ref_of(t, s, a, L);
      ++n3;
    }
    for (int a = 1; a < L; ++a)
      for (int b = a + 1; b < L; ++b) {
        t.v4[i][n4][0] = ref_of(t, s, 0, a);
        t.v4[i][n4][1] = ref_of(t, s, a, b);
        t.v4[i][n4][2] = ref_of(t, s, b, L);
        ++n4;
      }
    t.nv3[i] = n3;
    t.nv4[i] = n4;
  }
  for (int code = 0; code < ipow(K, K); ++code) {
    int s[5] = {};
    if (!tuple_of(K, K, code, s)) continue;
    const int c = t.ncol++;
    for (int k = 0; k < K; ++k) t.perm[c][k] = s[k];
    int l = 0;
    if (c > 0)
      while (l < K && t.perm[c - 1][l] == s[l]) ++l;
    t.lcp[c] = l;
    for (int m = 0; m < K; ++m) t.pmask[c][m] = mask_of(s, 0, m);
    for (int j = 0; j < K; ++j)
      for (int m = j + 1; m <= K; ++m)
        if (!(j == 0 && m == K)) t.sub[c][j][m] = ref_of(t, s, j, m);
    if (s[0] < s[K - 1]) {
      const int f = t.nfull++;
      t.fidx[c] = f;
      int n3 = 0, n4 = 0;
      for (int a = 1; a < K; ++a) {
        t.fv3[f][n3][0] = ref_of(t, s, 0, a);
        t.fv3[f][n3][1] = ref_of(t, s, a, K);
        ++n3;
      }
      for (int a = 1; a < K; ++a)
        for (int b = a + 1; b < K; ++b) {
          t.fv4[f][n4][0] = ref_of(t, s, 0, a);
          t.fv4[f][n4][1] = ref_of(t, s, a, b);
          t.fv4[f][n4][2] = ref_of(t, s, b, K);
          ++n4;
        }
      t.fnv3[f] = n3;
      t.fnv4[f] = n4;
    }
  }
  // non-canonical orderings point at their reverse (which precedes them lexicographically)
  for (int c = 0; c < t.ncol; ++c) {
    const int* s = t.perm[c];
    if (s[0] < s[K - 1]) continue;
    for (int d = 0; d < t.ncol; ++d) {
      bool rev = true;
      for (int k = 0; k < K; ++k)
        if (t.perm[d][k] != s[K - 1 - k]) rev = false;
      if (rev) t.fidx[c] = -t.fidx[d] - 1;
    }
  }
  return t;
}

template <int K>
struct Tables {
  static constexpr Tab t = make_tab(K);
};

// accessors usable in constant expressions of device code
template <int K> __host__ __device__ constexpr int nseq() { return Tables<K>::t.nseq; }
template <int K> __host__ __device__ constexpr int ncol() { return Tables<K>::t.ncol; }
template <int K> __host__ __device__ constexpr int nfull() { return Tables<K>::t.nfull; }
template <int K> __host__ __device__ constexpr int smask(int s) { return Tables<K>::t.mask[s]; }
template <int K> __host__ __device__ constexpr int nv3(int s) { return Tables<K>::t.nv3[s]; }
template <int K> __host__ __device__ constexpr int nv4(int s) { return Tables<K>::t.nv4[s]; }
template <int K> __host__ __device__ constexpr int v3(int s, int k, int i) { return Tables<K>::t.v3[s][k][i]; }
template <int K> __host__ __device__ constexpr int v4(int s, int k, int i) { return Tables<K>::t.v4[s][k][i]; }
template <int K> __host__ __device__ constexpr int lcp(int c) { return Tables<K>::t.lcp[c]; }
template <int K> __host__ __device__ constexpr int pmask(int c, int m) { return Tables<K>::t.pmask[c][m]; }
template <int K> __host__ __device__ constexpr int sub(int c, int j, int m) { return Tables<K>::t.sub[c][j][m]; }
template <int K> __host__ __device__ constexpr int fidx(int c) { return Tables<K>::t.fidx[c]; }
template <int K> __host__ __device__ constexpr int fnv3(int f) { return Tables<K>::t.fnv3[f]; }
template <int K> __host__ __device__ constexpr int fnv4(int f) { return Tables<K>::t.fnv4[f]; }
template <int K> __host__ __device__ constexpr int fv3(int f, int k, int i) { return Tables<K>::t.fv3[f][k][i]; }
template <int K> __host__ __device__ constexpr int fv4(int f, int k, int i) { return Tables<K>::t.fv4[f][k][i]; }

}  // namespace st
}  // namespace mg
