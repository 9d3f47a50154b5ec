"""The compile-time recursion tables (csrc/mg_static_tables.h, which drive the unrolled FP32 kernels)
equal the run-time ones (csrc/mg_tables.cpp, which drive the other kernels) entry by entry, for
K = 2..5 gluons: both are compiled here with the host compiler into a small checker."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2210_11122_gb300", "csrc")

CHECKER = r'''
#define __host__
#define __device__
#include <cstdio>
#include "mg_internal.h"
#include "mg_static_tables.h"

template <int K> int check() {
  mg::Tables t;
  mg::build_tables(K, t);
  constexpr const mg::st::Tab& s = mg::st::Tables<K>::t;
  int bad = 0;
  auto eq = [&](long a, long b, const char* what, int i) { if (a != b) { ++bad; std::printf("K=%d %s[%d]: %ld != %ld\n", K, what, i, a, b); } };
  eq(s.nseq, t.nseq, "nseq", 0); eq(s.ncol, t.ncol, "ncol", 0); eq(s.nfull, t.nfull, "nfull", 0);
  for (int i = 0; i < t.nseq; ++i) {
    eq(s.len[i], t.seq_len[i], "len", i); eq(s.mask[i], t.seq_mask[i], "mask", i);
    eq(s.nv3[i], t.seq_nv3[i], "nv3", i); eq(s.nv4[i], t.seq_nv4[i], "nv4", i);
    for (int k = 0; k < t.seq_nv3[i]; ++k) for (int j = 0; j < 2; ++j) eq(s.v3[i][k][j], t.seq_v3[i][k][j], "v3", i);
    for (int k = 0; k < t.seq_nv4[i]; ++k) for (int j = 0; j < 3; ++j) eq(s.v4[i][k][j], t.seq_v4[i][k][j], "v4", i);
  }
  for (int c = 0; c < t.ncol; ++c) {
    eq(s.lcp[c], t.lcp[c], "lcp", c); eq(s.fidx[c], t.full_idx[c], "fidx", c);
    for (int g = 0; g < K; ++g) { eq(s.perm[c][g], t.perm[c][g], "perm", c); eq(s.pmask[c][g], t.prefix_mask[c][g], "pmask", c); }
    for (int j = 0; j < K; ++j) for (int m = j + 1; m <= K; ++m) if (!(j == 0 && m == K)) eq(s.sub[c][j][m], t.sub[c][j][m], "sub", c);
  }
  for (int f = 0; f < t.nfull; ++f) {
    eq(s.fnv3[f], t.full_nv3[f], "fnv3", f); eq(s.fnv4[f], t.full_nv4[f], "fnv4", f);
    for (int k = 0; k < t.full_nv3[f]; ++k) for (int j = 0; j < 2; ++j) eq(s.fv3[f][k][j], t.full_v3[f][k][j], "fv3", f);
    for (int k = 0; k < t.full_nv4[f]; ++k) for (int j = 0; j < 3; ++j) eq(s.fv4[f][k][j], t.full_v4[f][k][j], "fv4", f);
  }
  return bad;
}

int main() {
  const int bad = check<2>() + check<3>() + check<4>() + check<5>();
  std::printf("mismatches %d\n", bad);
  return bad == 0 ? 0 : 1;
}
'''


def test_compile_time_tables_equal_run_time_tables(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "check_tables.cpp"
    src.write_text(CHECKER)
    exe = tmp_path / "check_tables"
    cmd = [cxx, "-std=c++17", "-O1", "-fconstexpr-ops-limit=1000000000", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
           str(src), os.path.join(CSRC, "mg_tables.cpp"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout[-3000:]
    assert "mismatches 0" in r.stdout
