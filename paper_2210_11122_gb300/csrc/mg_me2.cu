// mg_me2.cu -- matrix-element kernel, one thread per (event, gluon-helicity combination).
//
// Same physics as the per-helicity kernel of mg_me.cu (HELAS wavefunctions, every tree diagram of
// g g -> t tbar + (K-2) g summed into colour-ordered amplitudes by the Berends-Giele recursion of
// mg_tables.cpp, exact colour matrix, helicity sum; the hot path of the paper's Sec. 2), organised
// for GB300's FP64 pipe (2 DFMA/clk/SM, 1/64 of FP32), where the instruction count is the cost:
//   * the gluon currents J(seq) and the all-gluon currents J(sigma) depend only on the gluon
//     helicities: one thread computes them once and reuses them for the 4 top-helicity pairs;
//   * quark-line prefixes depend on the top helicity only: one depth-first walk per top helicity,
//     each leaf forming the amplitudes of both antitop helicities;
//   * (gamma.J) v is precomputed per antitop helicity for every gluon current;
//   * every complex product-accumulate is an FMA chain; the quark propagator factor
//     -g/(Q^2 - m^2) is folded into the coefficients of (Qslash + m) once per event subset.
// Output: per slot (gluon combination) the colour-summed |M_h|^2 summed over its good top
// helicities, or (filter mode) |M_h|^2 of every helicity h separately.
#include <cuda_runtime.h>

#include "mg_internal.h"
#include "mg_kernels.h"
#include "mg_me_algebra.cuh"

namespace mg {
namespace v2 {

// One thread per event: the event's record, AoSoA (page of 32 events, value-major within a page).
// repair != NULL: events whose smallest internal invariant |P^2| or |Q^2 - m^2| (over the gluon and
// quark propagators of the recursion) is below cst.fp32_tau * s are appended to repair[] (count in
// *nrepair): FP32 rounding is amplified ~ 1/sqrt(invariant/s) there (collinear and soft gluons).
template <int K, class T>
__global__ void __launch_bounds__(128) k_event_prep(const double* __restrict__ mom, int64_t nevt, MeConst cst,
                                                    T* __restrict__ rec, int* __restrict__ repair,
                                                    int* __restrict__ nrepair, uint8_t* __restrict__ flag) {
  constexpr int npar = K + 2, NSUB = 1 << K;
  using L = EvLayout<K>;
  const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (e >= nevt) return;
  double p[npar][4];
  const double* base = mom + (e / kPage) * npar * 4 * kPage + (e % kPage);
#pragma unroll
  for (int i = 0; i < npar; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) p[i][m] = __ldg(base + (i * 4 + m) * kPage);
  T PT[NSUB][4], gprop[NSUB], qc[NSUB][5], pol[K][5];
  cx<T> ub[2][4], vv[2][4];
  double xmin = 1.0;
  event_data<K, T>(p, cst, PT, gprop, qc, pol, ub, vv, &xmin);
  const bool redo = repair && xmin < cst.fp32_tau;
  if (redo) repair[atomicAdd(nrepair, 1)] = static_cast<int>(e);
  if (flag) flag[e] = redo ? 1 : 0;
  T* out = rec + (e / kPage) * L::NITEM * kPage + (e % kPage);
#pragma unroll
  for (int S = 0; S < NSUB; ++S) {
#pragma unroll
    for (int m = 0; m < 4; ++m) out[(L::PT + 4 * S + m) * kPage] = PT[S][m];
    out[(L::GP + S) * kPage] = gprop[S];
#pragma unroll
    for (int c = 0; c < 5; ++c) out[(L::QC + 5 * S + c) * kPage] = qc[S][c];
  }
#pragma unroll
  for (int g = 0; g < K; ++g)
#pragma unroll
    for (int i = 0; i < 5; ++i) out[(L::EPS + 5 * g + i) * kPage] = pol[g][i];
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      out[(L::UB + (l * 4 + a) * 2) * kPage] = ub[l][a].r;
      out[(L::UB + (l * 4 + a) * 2 + 1) * kPage] = ub[l][a].i;
      out[(L::VV + (l * 4 + a) * 2) * kPage] = vv[l][a].r;
      out[(L::VV + (l * 4 + a) * 2 + 1) * kPage] = vv[l][a].i;
    }
}

// JOUT: instead of colour sums, write the jamps of every helicity of the slot as FP32 complex
// numbers to jout[((e * 4 * 2^K) + slot * 4 + 2 * top + antitop) * ncol + sigma] (zeros for helicities
// outside the mask), for the tensor-core colour sum.
template <int K, class T, bool PER_HEL, bool PREP, bool JOUT>
__global__ void __launch_bounds__(kMeThreads)
k_me_gluonhel(const double* __restrict__ mom, const T* __restrict__ rec, int64_t nevt, const Tables* __restrict__ tab,
              const int* __restrict__ gslots, const int* __restrict__ nslot_dev, const uint32_t* __restrict__ mask,
              const T* __restrict__ ctri, MeConst cst, double* __restrict__ out, int64_t stride,
              float2* __restrict__ jout, int tile_ev, int slot_major, const int* __restrict__ evlist,
              const int* __restrict__ nlist, int rows_out, const uint8_t* __restrict__ skip) {
  constexpr int npar = K + 2;
  constexpr int NSEQ = Sizes<K>::nseq;
  constexpr int NCOL = Sizes<K>::ncol;
  constexpr int NFULL = Sizes<K>::nfull;
  constexpr int NSUB = 1 << K;
  const int tile_sl = kMeThreads / tile_ev;
  const unsigned bev = slot_major ? blockIdx.y : blockIdx.x, bsl = slot_major ? blockIdx.x : blockIdx.y;
  const int64_t et = static_cast<int64_t>(bev) * tile_ev + threadIdx.x % tile_ev;
  const int slot = static_cast<int>(bsl) * tile_sl + static_cast<int>(threadIdx.x) / tile_ev;
  if (et >= nevt || slot >= *nslot_dev) return;
  // evlist: the thread works on event evlist[et] of the batch (et < *nlist), else on event et
  if (evlist && et >= *nlist) return;
  const int64_t e = evlist ? static_cast<int64_t>(evlist[et]) : et;
  if (PREP && skip && skip[e]) return;   // recomputed by another launch
  const int gc = gslots[slot];   // bit g = helicity (+1) of gluon g

  const T gs = static_cast<T>(cst.gs);
  T PT[NSUB][4];
  T gprop[NSUB];
  T qc[NSUB][5];
  cx<T> J[NSEQ][4];
  cx<T> ub[2][4], vv[2][4];
  if (PREP) {
    using L = EvLayout<K>;
    const T* in = rec + (e / kPage) * L::NITEM * kPage + (e % kPage);
#pragma unroll
    for (int S = 0; S < NSUB; ++S) {
#pragma unroll
      for (int m = 0; m < 4; ++m) PT[S][m] = __ldg(in + (L::PT + 4 * S + m) * kPage);
      gprop[S] = __ldg(in + (L::GP + S) * kPage);
#pragma unroll
      for (int c = 0; c < 5; ++c) qc[S][c] = __ldg(in + (L::QC + 5 * S + c) * kPage);
    }
#pragma unroll
    for (int g = 0; g < K; ++g) {
      T pol[5];
#pragma unroll
      for (int i = 0; i < 5; ++i) pol[i] = __ldg(in + (L::EPS + 5 * g + i) * kPage);
      ext_gluon(pol, (gc >> g) & 1 ? 1 : -1, g >= 2, J[g]);
    }
#pragma unroll
    for (int l = 0; l < 2; ++l)
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        ub[l][a] = {__ldg(in + (L::UB + (l * 4 + a) * 2) * kPage), __ldg(in + (L::UB + (l * 4 + a) * 2 + 1) * kPage)};
        vv[l][a] = {__ldg(in + (L::VV + (l * 4 + a) * 2) * kPage), __ldg(in + (L::VV + (l * 4 + a) * 2 + 1) * kPage)};
      }
  } else {
    double p[npar][4];
    const double* base = mom + (e / kPage) * npar * 4 * kPage + (e % kPage);
#pragma unroll
    for (int i = 0; i < npar; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) p[i][m] = __ldg(base + (i * 4 + m) * kPage);
    T pol[K][5];
    event_data<K, T>(p, cst, PT, gprop, qc, pol, ub, vv);
#pragma unroll
    for (int g = 0; g < K; ++g) ext_gluon(pol[g], (gc >> g) & 1 ? 1 : -1, g >= 2, J[g]);
  }

  // ---- gluon currents (helicities of gc) ----
  for (int s = K; s < NSEQ; ++s) {
    cx<T> acc[4] = {};
    const int n3 = tab->seq_nv3[s];
    for (int k = 0; k < n3; ++k) {
      const int16_t rl = tab->seq_v3[s][k][0], rr = tab->seq_v3[s][k][1];
      const int il = rslot(rl), ir = rslot(rr);
      v3_acc(acc, J[il], J[ir], PT[tab->seq_mask[il]], PT[tab->seq_mask[ir]], rneg(rl) != rneg(rr));
    }
    const int n4 = tab->seq_nv4[s];
    for (int k = 0; k < n4; ++k) {
      const int16_t ra = tab->seq_v4[s][k][0], rb = tab->seq_v4[s][k][1], rc = tab->seq_v4[s][k][2];
      v4_acc(acc, J[rslot(ra)], J[rslot(rb)], J[rslot(rc)], gs, rneg(ra) ^ rneg(rb) ^ rneg(rc));
    }
    const T f = gprop[tab->seq_mask[s]];
#pragma unroll
    for (int m = 0; m < 4; ++m) J[s][m] = cscale(f, acc[m]);
  }
  // all gluons on one current (canonical orderings)
  cx<T> JF[NFULL][4];
  for (int f = 0; f < NFULL; ++f) {
    cx<T> acc[4] = {};
    const int n3 = tab->full_nv3[f];
    for (int k = 0; k < n3; ++k) {
      const int16_t rl = tab->full_v3[f][k][0], rr = tab->full_v3[f][k][1];
      const int il = rslot(rl), ir = rslot(rr);
      v3_acc(acc, J[il], J[ir], PT[tab->seq_mask[il]], PT[tab->seq_mask[ir]], rneg(rl) != rneg(rr));
    }
    const int n4 = tab->full_nv4[f];
    for (int k = 0; k < n4; ++k) {
      const int16_t ra = tab->full_v4[f][k][0], rb = tab->full_v4[f][k][1], rc = tab->full_v4[f][k][2];
      v4_acc(acc, J[rslot(ra)], J[rslot(rb)], J[rslot(rc)], gs, rneg(ra) ^ rneg(rb) ^ rneg(rc));
    }
    const T fz = gprop[NSUB - 1];
#pragma unroll
    for (int m = 0; m < 4; ++m) JF[f][m] = cscale(fz, acc[m]);
  }

  // ---- antitop spinors and (gamma.J) v for both antitop helicities ----
  // (gamma.J) v for every current and both antitop helicities: precomputed in FP64 (saves FP64
  // instructions); in FP32 each jamp term forms ubar-side (row spinor x gamma.J) on the fly instead,
  // keeping 2 NSEQ spinors out of the thread's local memory (FP32 arithmetic is cheap, memory is not).
  constexpr bool kTableX = sizeof(T) == 8;
  cx<T> X[kTableX ? 2 : 1][kTableX ? NSEQ : 1][4];
  if (kTableX) {
#pragma unroll
    for (int b = 0; b < 2; ++b)
      for (int s = 0; s < NSEQ; ++s) gamma_col(J[s], vv[b], X[b][s]);
  }

  // helicity index of (gc, top helicity a, antitop helicity b)
  int hbase = 0;
#pragma unroll
  for (int g = 0; g < K; ++g)
    if ((gc >> g) & 1) hbase |= 1 << (npar - 1 - (g < 2 ? g : g + 2));
  const int bit_t = 1 << (npar - 3), bit_tb = 1 << (npar - 4);

  double total = 0.0;
  for (int a = 0; a < 2; ++a) {
    const int h0 = hbase | (a ? bit_t : 0), h1 = h0 | bit_tb;
    const bool good0 = PER_HEL || ((mask[h0 >> 5] >> (h0 & 31)) & 1u);
    const bool good1 = PER_HEL || ((mask[h1 >> 5] >> (h1 & 31)) & 1u);
    if (!good0 && !good1) {
      if (JOUT) {
        float2* row = jout + (e * (4 << K) + slot * 4 + 2 * a) * NCOL;
        for (int c = 0; c < 2 * NCOL; ++c) row[c] = make_float2(0.f, 0.f);
      }
      continue;
    }
    cx<T> stk[K][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) stk[0][q] = ub[a][q];
    cx<T> Jq[2][4];
    quark_current(stk[0], vv[0], Jq[0]);
    quark_current(stk[0], vv[1], Jq[1]);
    cx<T> A[2][NCOL];
    for (int c = 0; c < NCOL; ++c) {
      const int l = tab->lcp[c];
      for (int m = l + 1; m < K; ++m) {
        cx<T> acc[4] = {};
        for (int j = 0; j < m; ++j) {
          const int16_t r = tab->sub[c][j][m];
          row_gamma_acc(acc, stk[j], J[rslot(r)], rneg(r));
        }
        row_prop(acc, qc[tab->prefix_mask[c][m]], stk[m]);
      }
      const int fi = tab->full_idx[c];
      const int fidx = fi >= 0 ? fi : -fi - 1;
      const bool fneg = fi < 0 && !(K & 1);   // reflection sign (-1)^(K+1)
      if (kTableX) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          cx<T> amp = mdot(Jq[b], JF[fidx]);   // all gluons on one current: ubar gamma.J v = Jq.J
          if (fneg) amp = cneg(amp);
          for (int j = 1; j < K; ++j) {
            const int16_t r = tab->sub[c][j][K];
            sdot_acc(amp, stk[j], X[b][rslot(r)], rneg(r));
          }
          A[b][c] = amp;
        }
      } else {
        cx<T> amp0 = mdot(Jq[0], JF[fidx]), amp1 = mdot(Jq[1], JF[fidx]);
        if (fneg) { amp0 = cneg(amp0); amp1 = cneg(amp1); }
        for (int j = 1; j < K; ++j) {
          const int16_t r = tab->sub[c][j][K];
          cx<T> t[4] = {};
          row_gamma_acc(t, stk[j], J[rslot(r)], rneg(r));
          sdot_acc(amp0, t, vv[0], false);
          sdot_acc(amp1, t, vv[1], false);
        }
        A[0][c] = amp0;
        A[1][c] = amp1;
      }
    }
    if constexpr (JOUT) {
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const bool good = b ? good1 : good0;
        float2* row = jout + (e * (4 << K) + slot * 4 + 2 * a + b) * NCOL;
        for (int c = 0; c < NCOL; ++c)
          row[c] = good ? make_float2(static_cast<float>(A[b][c].r), static_cast<float>(A[b][c].i)) : make_float2(0.f, 0.f);
      }
      continue;
    } else {
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int h = b ? h1 : h0;
        const bool good = b ? good1 : good0;
        if (!good) continue;
        const double v = static_cast<double>(colour_sum<NCOL, T>(A[b], ctri)) * cst.colour_scale;
        if (PER_HEL) out[h * stride + e] = v;
        else total += v;
      }
    }
  }
  if (!PER_HEL && !JOUT) {
    if (rows_out) {   // tensor-core row layout: slot*4 + (2 top + antitop); the slot total in the first row
      out[(slot * 4) * stride + e] = total;
      out[(slot * 4 + 1) * stride + e] = 0.0;
      out[(slot * 4 + 2) * stride + e] = 0.0;
      out[(slot * 4 + 3) * stride + e] = 0.0;
    } else {
      out[slot * stride + e] = total;
    }
  }
}

// Gluon-helicity combinations with at least one good helicity (fixed ascending order).
__global__ void k_gluon_slots(const uint32_t* __restrict__ mask, int K, int* __restrict__ gslots, int* __restrict__ n,
                              int* __restrict__ nrows) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int npar = K + 2;
  int cnt = 0;
  for (int gc = 0; gc < (1 << K); ++gc) {
    int hb = 0;
    for (int g = 0; g < K; ++g)
      if ((gc >> g) & 1) hb |= 1 << (npar - 1 - (g < 2 ? g : g + 2));
    bool any = false;
    for (int t = 0; t < 4; ++t) {
      const int h = hb | ((t & 1) << (npar - 3)) | ((t >> 1) << (npar - 4));
      any = any || ((mask[h >> 5] >> (h & 31)) & 1u);
    }
    if (any) gslots[cnt++] = gc;
  }
  *n = cnt;
  *nrows = 4 * cnt;
}

}  // namespace v2

cudaError_t launch_gluon_slots(const uint32_t* mask, int K, int* gslots, int* n, int* nrows, cudaStream_t st) {
  v2::k_gluon_slots<<<1, 32, 0, st>>>(mask, K, gslots, n, nrows);
  return cudaGetLastError();
}

template <int K, class T, bool PER_HEL>
static cudaError_t launch_v2(const double* mom, void* prep, int64_t nevt, const Tables* tab, const int* gslots,
                             int maxslot, const int* nslot, const uint32_t* mask, const void* ctri_any,
                             const MeConst& cst, double* out, int64_t stride, float2* jout, MeShape shape,
                             const uint8_t* skip, const int* evlist, const int* nlist, int rows_out, cudaStream_t st) {
  const T* ctri = static_cast<const T*>(ctri_any);
  int tev = shape.tile_ev;
  if (tev != 32 && tev != 64 && tev != 128) tev = 128;
  const int tsl = kMeThreads / tev;
  const unsigned nev_t = static_cast<unsigned>((nevt + tev - 1) / tev), nsl_t = static_cast<unsigned>((maxslot + tsl - 1) / tsl);
  const int sm = shape.slot_major ? 1 : 0;
  dim3 grid = sm ? dim3(nsl_t, nev_t) : dim3(nev_t, nsl_t);
  if (nev_t == 0 || nsl_t == 0) return cudaSuccess;
  if (prep && !PER_HEL) {
    const T* rec = static_cast<const T*>(prep);
    if (shape.unrolled && me_static_available(K, sizeof(T) == 4))
      return launch_me_static(K, sizeof(T) == 4, rec, nevt, gslots, maxslot, nslot, mask, cst, out, stride, jout, shape,
                              skip, st);
    if (jout)
      v2::k_me_gluonhel<K, T, false, true, true><<<grid, kMeThreads, 0, st>>>(mom, rec, nevt, tab, gslots, nslot, mask,
                                                                             ctri, cst, out, stride, jout, tev, sm, nullptr,
                                                                             nullptr, 0, skip);
    else
      v2::k_me_gluonhel<K, T, false, true, false><<<grid, kMeThreads, 0, st>>>(mom, rec, nevt, tab, gslots, nslot,
                                                                              mask, ctri, cst, out, stride, nullptr, tev,
                                                                              sm, nullptr, nullptr, 0, skip);
  } else {
    v2::k_me_gluonhel<K, T, PER_HEL, false, false><<<grid, kMeThreads, 0, st>>>(mom, nullptr, nevt, tab, gslots, nslot,
                                                                                 mask, ctri, cst, out, stride, nullptr,
                                                                                 tev, sm, evlist, nlist, rows_out,
                                                                                 nullptr);
  }
  return cudaGetLastError();
}

template <int K, class T>
static cudaError_t launch_prep(const double* mom, int64_t nevt, const MeConst& cst, void* rec, int* repair,
                               int* nrepair, uint8_t* flag, cudaStream_t st) {
  if (nevt <= 0) return cudaSuccess;
  v2::k_event_prep<K, T><<<static_cast<unsigned>((nevt + 127) / 128), 128, 0, st>>>(mom, nevt, cst, static_cast<T*>(rec),
                                                                                   repair, nrepair, flag);
  return cudaGetLastError();
}

cudaError_t launch_event_prep(int K, bool fp32, const double* mom, int64_t nevt, const MeConst& cst, void* rec,
                              int* repair, int* nrepair, uint8_t* flag, cudaStream_t st) {
  switch (K) {
    case 2: return fp32 ? launch_prep<2, float>(mom, nevt, cst, rec, repair, nrepair, flag, st)
                        : launch_prep<2, double>(mom, nevt, cst, rec, repair, nrepair, flag, st);
    case 3: return fp32 ? launch_prep<3, float>(mom, nevt, cst, rec, repair, nrepair, flag, st)
                        : launch_prep<3, double>(mom, nevt, cst, rec, repair, nrepair, flag, st);
    case 4: return fp32 ? launch_prep<4, float>(mom, nevt, cst, rec, repair, nrepair, flag, st)
                        : launch_prep<4, double>(mom, nevt, cst, rec, repair, nrepair, flag, st);
    case 5: return fp32 ? launch_prep<5, float>(mom, nevt, cst, rec, repair, nrepair, flag, st)
                        : launch_prep<5, double>(mom, nevt, cst, rec, repair, nrepair, flag, st);
    default: return cudaErrorInvalidValue;
  }
}

int64_t event_record_bytes(int K, bool fp32) {
  int nitem = 0;
  switch (K) {
    case 2: nitem = v2::EvLayout<2>::NITEM; break;
    case 3: nitem = v2::EvLayout<3>::NITEM; break;
    case 4: nitem = v2::EvLayout<4>::NITEM; break;
    case 5: nitem = v2::EvLayout<5>::NITEM; break;
    default: return 0;
  }
  return static_cast<int64_t>(nitem) * (fp32 ? 4 : 8);
}

cudaError_t launch_me_gluonhel(int K, bool fp32, bool per_hel, const double* mom, void* prep, int64_t nevt,
                               const Tables* tab, const int* gslots, int maxslot, const int* nslot,
                               const uint32_t* mask, const double* ctri64, const float* ctri32, const MeConst& cst,
                               double* out, int64_t stride, cudaStream_t st, float2* jout, MeShape shape,
                               const uint8_t* skip, const int* evlist, const int* nlist, int rows_out) {
#define MG_V2_CASE(KK)                                                                                              \
  case KK:                                                                                                          \
    if (per_hel) return fp32 ? launch_v2<KK, float, true>(mom, prep, nevt, tab, gslots, maxslot, nslot, mask, ctri32, cst,  \
                                                          out, stride, jout, shape, skip, evlist, nlist, rows_out, st)                                          \
                             : launch_v2<KK, double, true>(mom, prep, nevt, tab, gslots, maxslot, nslot, mask, ctri64, cst, \
                                                           out, stride, jout, shape, skip, evlist, nlist, rows_out, st);                                        \
    return fp32 ? launch_v2<KK, float, false>(mom, prep, nevt, tab, gslots, maxslot, nslot, mask, ctri32, cst, out, stride, \
                                              jout, shape, skip, evlist, nlist, rows_out, st)                                                                   \
                : launch_v2<KK, double, false>(mom, prep, nevt, tab, gslots, maxslot, nslot, mask, ctri64, cst, out, stride,\
                                               jout, shape, skip, evlist, nlist, rows_out, st);
  switch (K) {
    MG_V2_CASE(2)
    MG_V2_CASE(3)
    MG_V2_CASE(4)
    MG_V2_CASE(5)
    default: return cudaErrorInvalidValue;
  }
#undef MG_V2_CASE
}

}  // namespace mg
