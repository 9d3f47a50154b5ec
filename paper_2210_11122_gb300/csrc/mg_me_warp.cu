// mg_me_warp.cu -- FP32 matrix-element kernel with one lane group (a warp or part of one) per (event,
// gluon-helicity slot).
//
// Same physics, record input and outputs as the per-thread kernels (mg_me_kernel.cuh, mg_me3.cu), for
// processes whose per-slot state does not fit in a thread: with 5 gluons a slot carries 105 gluon
// currents, 60 all-gluon currents and 4 x 120 jamps (~9 KB), which a thread can only keep in local
// memory (spilled to L2 and DRAM at the occupancy the FP32 pipe needs).  Here the G lanes of a group
// (G = 32 for 5 gluons, 8 for 4, 4 for 3) share that state in shared memory and split the work:
//   * currents level by level (all sequences of one length are independent): one sequence per lane;
//   * the quark-line walk: the first half of the group takes top helicity -, the second half top
//     helicity +, each lane a contiguous run of colour orderings (prefix spinors shared along the run,
//     in registers);
//   * the colour sums of the four helicities together: rows of C A per lane (register-blocked over
//     rows and helicities), then sums over the group; or (jamp output) the jamps are written out for
//     the tensor-core colour sum.
#include <cuda_runtime.h>

#include "mg_internal.h"
#include "mg_kernels.h"
#include "mg_me_algebra.cuh"

namespace mg {
namespace wk {

using v2::cx;

constexpr int kWarps = 4;   // warps per block; a block holds slots of one event

// lanes per slot G: the work of one slot spread over as many lanes as its widest stage keeps busy
template <int K> struct WSizes;
template <> struct WSizes<3> { static constexpr int ncol = 6, nseq = 6, nfull = 3, G = 4; };
template <> struct WSizes<4> { static constexpr int ncol = 24, nseq = 22, nfull = 12, G = 8; };
template <> struct WSizes<5> { static constexpr int ncol = 120, nseq = 105, nfull = 60, G = 32; };

// shared state of one slot: component-major, so that lanes reading different currents hit different banks
template <int K>
struct SlotState {
  float2 J[4][WSizes<K>::nseq];
  float2 JF[4][WSizes<K>::nfull];
  float2 A[4][WSizes<K>::ncol];   // jamps of helicity 2 * top + antitop
};

__device__ __forceinline__ cx<float> c2(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 f2(cx<float> v) { return make_float2(v.r, v.i); }

// first canonical sequence of length L (sequences are numbered by length: K singles, then L = 2, 3, ...)
__host__ __device__ constexpr int seq_start(int K, int L) {
  int s = K;
  for (int l = 2; l < L; ++l) {
    int n = 1;
    for (int i = 0; i < l; ++i) n *= K - i;
    s += n / 2;
  }
  return L <= 1 ? 0 : s;
}

template <int K, bool JOUT>
__global__ void __launch_bounds__(kWarps * 32)
k_me_warp(const float* __restrict__ rec, int64_t nevt, const Tables* __restrict__ tab, const int* __restrict__ gslots,
          const int* __restrict__ nslot_dev, const uint32_t* __restrict__ mask, const float* __restrict__ cfull,
          MeConst cst, double* __restrict__ out, int64_t stride, float2* __restrict__ jout,
          const uint8_t* __restrict__ skip) {
  using L = v2::EvLayout<K>;
  constexpr int npar = K + 2, NCOL = WSizes<K>::ncol, NFULL = WSizes<K>::nfull;
  constexpr int NSUB = 1 << K;
  constexpr int G = WSizes<K>::G, GPW = 32 / G;   // lanes per slot, slots per warp
  __shared__ SlotState<K> sh[kWarps * GPW];
  const int warp = threadIdx.x >> 5, grp = (threadIdx.x & 31) / G, lane = threadIdx.x % G;
  const unsigned gmask = (G == 32 ? 0xffffffffu : ((1u << (G & 31)) - 1u)) << (grp * G);   // this group's lanes
  const int64_t e = blockIdx.x;
  const int slot = (blockIdx.y * kWarps + warp) * GPW + grp;
  if (e >= nevt || slot >= *nslot_dev) return;   // whole groups leave: every sync below is per group
  if (skip && skip[e]) return;   // recomputed by another launch
  SlotState<K>& S = sh[warp * GPW + grp];
  const int gc = gslots[slot];   // bit g = helicity (+1) of gluon g
  const float* in = rec + (e / kPage) * L::NITEM * kPage + (e % kPage);
  auto ld = [&](int item) -> float { return __ldg(in + item * kPage); };
  const float gs = static_cast<float>(cst.gs);

  // ---- external gluon currents ----
  if (lane < K) {
    float pol[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) pol[i] = ld(L::EPS + 5 * lane + i);
    cx<float> w[4];
    v2::ext_gluon(pol, (gc >> lane) & 1 ? 1 : -1, lane >= 2, w);
#pragma unroll
    for (int m = 0; m < 4; ++m) S.J[m][lane] = f2(w[m]);
  }
  __syncwarp(gmask);
  auto getJ = [&](int slot_ref, cx<float>* j) {
#pragma unroll
    for (int m = 0; m < 4; ++m) j[m] = c2(S.J[m][slot_ref >> 1]);
  };
  auto getP = [&](int seq, float* P) {
    const int msk = tab->seq_mask[seq];
#pragma unroll
    for (int m = 0; m < 4; ++m) P[m] = ld(L::PT + 4 * msk + m);
  };
  // current of sequence s (splits from the tables) into acc
  auto current = [&](int nv3, const int16_t (*v3)[2], int nv4, const int16_t (*v4)[3], cx<float>* acc) {
    for (int k = 0; k < nv3; ++k) {
      const int rl = v3[k][0], rr = v3[k][1];
      cx<float> JL[4], JR[4];
      float PL[4], PR[4];
      getJ(rl, JL);
      getJ(rr, JR);
      getP(rl >> 1, PL);
      getP(rr >> 1, PR);
      v2::v3_acc(acc, JL, JR, PL, PR, ((rl ^ rr) & 1) != 0);
    }
    for (int k = 0; k < nv4; ++k) {
      const int ra = v4[k][0], rb = v4[k][1], rc = v4[k][2];
      cx<float> JA[4], JB[4], JC[4];
      getJ(ra, JA);
      getJ(rb, JB);
      getJ(rc, JC);
      v2::v4_acc(acc, JA, JB, JC, gs, ((ra ^ rb ^ rc) & 1) != 0);
    }
  };

  // ---- gluon currents by length: the sequences of one length are independent ----
#pragma unroll
  for (int len = 2; len < K; ++len) {
    for (int s = seq_start(K, len) + lane; s < seq_start(K, len + 1); s += G) {
      cx<float> acc[4] = {};
      current(tab->seq_nv3[s], tab->seq_v3[s], tab->seq_nv4[s], tab->seq_v4[s], acc);
      const float f = ld(L::GP + tab->seq_mask[s]);
#pragma unroll
      for (int m = 0; m < 4; ++m) S.J[m][s] = f2(v2::cscale(f, acc[m]));
    }
    __syncwarp(gmask);
  }
  // ---- all gluons on one current (canonical orderings) ----
  {
    const float fz = ld(L::GP + NSUB - 1);
    for (int f = lane; f < NFULL; f += G) {
      cx<float> acc[4] = {};
      current(tab->full_nv3[f], tab->full_v3[f], tab->full_nv4[f], tab->full_v4[f], acc);
#pragma unroll
      for (int m = 0; m < 4; ++m) S.JF[m][f] = f2(v2::cscale(fz, acc[m]));
    }
  }
  __syncwarp(gmask);

  // ---- quark line: half-warp per top helicity, a run of orderings per lane ----
  int hbase = 0;
#pragma unroll
  for (int g = 0; g < K; ++g)
    if ((gc >> g) & 1) hbase |= 1 << (npar - 1 - (g < 2 ? g : g + 2));
  const int bit_t = 1 << (npar - 3), bit_tb = 1 << (npar - 4);
  bool good[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int h = hbase | ((k >> 1) ? bit_t : 0) | ((k & 1) ? bit_tb : 0);
    good[k] = (mask[h >> 5] >> (h & 31)) & 1u;
  }
  {
    constexpr int H = G / 2;   // lanes per top helicity
    const int a = lane / H, hl = lane % H;
    const int c0 = hl * NCOL / H, c1 = (hl + 1) * NCOL / H;
    if (good[2 * a] || good[2 * a + 1]) {
      cx<float> vv[2][4], stk[K][4], Jq[2][4];
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) vv[b][q] = {ld(L::VV + (b * 4 + q) * 2), ld(L::VV + (b * 4 + q) * 2 + 1)};
#pragma unroll
      for (int q = 0; q < 4; ++q) stk[0][q] = {ld(L::UB + (a * 4 + q) * 2), ld(L::UB + (a * 4 + q) * 2 + 1)};
      v2::quark_current(stk[0], vv[0], Jq[0]);
      v2::quark_current(stk[0], vv[1], Jq[1]);
      for (int c = c0; c < c1; ++c) {
        const int l = c == c0 ? 0 : tab->lcp[c];
#pragma unroll
        for (int m = 1; m < K; ++m) {
          if (m <= l) continue;
          cx<float> acc[4] = {};
#pragma unroll
          for (int j = 0; j < m; ++j) {
            const int r = tab->sub[c][j][m];
            cx<float> Jr[4];
            getJ(r, Jr);
            v2::row_gamma_acc(acc, stk[j], Jr, (r & 1) != 0);
          }
          const int pm = tab->prefix_mask[c][m];
          float q[5];
#pragma unroll
          for (int k = 0; k < 5; ++k) q[k] = ld(L::QC + 5 * pm + k);
          v2::row_prop(acc, q, stk[m]);
        }
        const int fi = tab->full_idx[c];
        const int fj = fi >= 0 ? fi : -fi - 1;
        const bool fneg = fi < 0 && !(K & 1);   // reflection sign (-1)^(K+1)
        cx<float> JFc[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) JFc[m] = c2(S.JF[m][fj]);
        cx<float> amp0 = v2::mdot(Jq[0], JFc), amp1 = v2::mdot(Jq[1], JFc);
        if (fneg) {
          amp0 = v2::cneg(amp0);
          amp1 = v2::cneg(amp1);
        }
#pragma unroll
        for (int j = 1; j < K; ++j) {
          const int r = tab->sub[c][j][K];
          cx<float> Jr[4], t[4] = {};
          getJ(r, Jr);
          v2::row_gamma_acc(t, stk[j], Jr, (r & 1) != 0);
          v2::sdot_acc(amp0, t, vv[0], false);
          v2::sdot_acc(amp1, t, vv[1], false);
        }
        S.A[2 * a][c] = good[2 * a] ? f2(amp0) : make_float2(0.f, 0.f);
        S.A[2 * a + 1][c] = good[2 * a + 1] ? f2(amp1) : make_float2(0.f, 0.f);
      }
    } else {
      for (int c = c0; c < c1; ++c) {
        S.A[2 * a][c] = make_float2(0.f, 0.f);
        S.A[2 * a + 1][c] = make_float2(0.f, 0.f);
      }
    }
  }
  __syncwarp(gmask);

  if constexpr (JOUT) {
    float2* row = jout + (e * (4 << K) + slot * 4) * NCOL;
    for (int i = lane; i < 4 * NCOL; i += G) row[i] = S.A[i / NCOL][i % NCOL];
  } else {
    // colour sums of the four helicities at once: lane l forms rows x = l, l + G, ... of w_h = C A_h
    // (C symmetric: row y of C read along x, coalesced; each C value feeds 8 FMAs), then A_h^* . w_h
    constexpr int XR = (NCOL + G - 1) / G;   // rows per lane
    float wr[4][XR] = {}, wi[4][XR] = {};
    for (int y = 0; y < NCOL; ++y) {
      float2 ay[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) ay[h] = S.A[h][y];
#pragma unroll
      for (int k = 0; k < XR; ++k) {
        const int x = lane + G * k;
        const float cxy = x < NCOL ? __ldg(cfull + y * NCOL + x) : 0.f;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          wr[h][k] = fmaf(cxy, ay[h].x, wr[h][k]);
          wi[h][k] = fmaf(cxy, ay[h].y, wi[h][k]);
        }
      }
    }
    double total = 0.0;
#pragma unroll
    for (int h = 0; h < 4; ++h) {   // jamps of helicities outside the mask are zero: no branch needed
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < XR; ++k) {
        const int x = lane + G * k;
        if (x < NCOL) {
          const float2 ax = S.A[h][x];
          s = fmaf(ax.x, wr[h][k], s);
          s = fmaf(ax.y, wi[h][k], s);
        }
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, G);
      if (good[h]) total += static_cast<double>(s) * cst.colour_scale;
    }
    if (lane == 0) out[slot * stride + e] = total;
  }
}

template <int K>
static cudaError_t launch_k(const void* rec, int64_t nevt, const Tables* tab, const int* gslots, int maxslot,
                            const int* nslot, const uint32_t* mask, const float* cfull, const MeConst& cst, double* out,
                            int64_t stride, float2* jout, const uint8_t* skip, cudaStream_t st) {
  if (nevt <= 0 || maxslot <= 0) return cudaSuccess;
  if (nevt > 0x7fffffffLL) return cudaErrorInvalidValue;
  constexpr int per_block = kWarps * (32 / WSizes<K>::G);   // slots per block
  const dim3 grid(static_cast<unsigned>(nevt), static_cast<unsigned>((maxslot + per_block - 1) / per_block));
  const float* r = static_cast<const float*>(rec);
  if (jout)
    k_me_warp<K, true><<<grid, kWarps * 32, 0, st>>>(r, nevt, tab, gslots, nslot, mask, cfull, cst, out, stride, jout,
                                                      skip);
  else
    k_me_warp<K, false><<<grid, kWarps * 32, 0, st>>>(r, nevt, tab, gslots, nslot, mask, cfull, cst, out, stride,
                                                       nullptr, skip);
  return cudaGetLastError();
}

}  // namespace wk

bool me_warp_available(int K, bool fp32) { return fp32 && K >= 3 && K <= 5; }

cudaError_t launch_me_warp(int K, const void* rec, int64_t nevt, const Tables* tab, const int* gslots, int maxslot,
                           const int* nslot, const uint32_t* mask, const float* cfull, const MeConst& cst, double* out,
                           int64_t stride, float2* jout, const uint8_t* skip, cudaStream_t st) {
  switch (K) {
    case 3: return wk::launch_k<3>(rec, nevt, tab, gslots, maxslot, nslot, mask, cfull, cst, out, stride, jout, skip, st);
    case 4: return wk::launch_k<4>(rec, nevt, tab, gslots, maxslot, nslot, mask, cfull, cst, out, stride, jout, skip, st);
    case 5: return wk::launch_k<5>(rec, nevt, tab, gslots, maxslot, nslot, mask, cfull, cst, out, stride, jout, skip, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mg
