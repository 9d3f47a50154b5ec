// mg_me_kernel.cuh -- the matrix-element kernel that reads the Berends-Giele recursion tables at run
// time, templated on the amplitude type: FP64 (the plain path), FP32, and double-float (dd::df, the
// FP32 modes' recomputation of events with a small internal invariant).  Instantiated in mg_me2.cu
// (FP64, FP32) and mg_me_dd.cu (double-float).
#pragma once

#include <type_traits>

#include "mg_me_algebra.cuh"

namespace mg {
namespace v2 {

__device__ constexpr int kFactorial[6] = {1, 1, 2, 6, 24, 120};

// The shared currents and quark-line prefixes of event e (FP64, share_stride doubles per event) are
// interleaved by page like the record: double d of the event sits at share_event(...)[d * kPage], so
// the 32 events of a warp read or write one 256-byte line per double
template <class P>
__device__ __forceinline__ P* share_event(P* share, int64_t e, int stride) {
  return share + (e / kPage) * static_cast<int64_t>(stride) * kPage + (e % kPage);
}

// JOUT: instead of colour sums, write the jamps of every helicity of the slot as FP32 complex
// numbers to jout[((e * 4 * 2^K) + slot * 4 + 2 * top + antitop) * ncol + sigma] (zeros for helicities
// outside the mask), for the tensor-core colour sum.
// SHARED (FP64 with a per-event record): the gluon currents of fewer than all gluons and their (gamma.J) v
// are not computed here but read from share where they are used (not copied into the thread's local
// memory), where k_share_level left them once per helicity assignment of their own gluons (item
// tab->share_base[s] + helicity bits of s's gluons, 24 doubles: J, then (gamma.J) v for both antitop
// helicities; page-interleaved, share_event); likewise the quark-line prefixes of k_prefix_level.
// LHE (FP64 with a per-event record, for the event-level epilogues): the colour sum of every helicity of
// the slot in its own row, out[(slot * 4 + 2 top + antitop) * stride + e] (zero for helicities outside
// the mask), and the slot's sum over its good helicities of every |jamp|^2,
// j2[(slot * ncol + sigma) * stride + e].
// The work of one thread: event e, gluon-helicity slot `slot` with gluon helicities gc (bit g = helicity +1
// of gluon g).  Called by k_me_gluonhel below and by the persistent multi-process kernel (mg_persist.cu).
template <int K, class T, bool PER_HEL, bool PREP, bool JOUT, bool SHARED = false, bool LHE = false>
__device__ __forceinline__ void me_slot(const double* __restrict__ mom, const T* __restrict__ rec, int64_t e, int slot,
                                        int gc, const Tables* __restrict__ tab, const uint32_t* __restrict__ mask,
                                        const typename ColourT<T>::type* __restrict__ ctri, const MeConst& cst,
                                        double* __restrict__ out, int64_t stride, float2* __restrict__ jout, int rows_out,
                                        const double* __restrict__ share, double* __restrict__ j2) {
  constexpr int npar = K + 2;
  constexpr int NSEQ = Sizes<K>::nseq;
  constexpr int NCOL = Sizes<K>::ncol;
  constexpr int NFULL = Sizes<K>::nfull;
  constexpr int NSUB = 1 << K;
  const T gs = static_cast<T>(cst.gs);
  // SHARED: the record's subset momenta, gluon propagators and quark-propagator coefficients are read
  // from the (page-interleaved) record where used, like the shared currents, not copied to local memory
  T PT[SHARED ? 1 : NSUB][4];
  T gprop[SHARED ? 1 : NSUB];
  T qc[SHARED ? 1 : NSUB][5];
  cx<T> J[SHARED ? 1 : NSEQ][4];   // SHARED: read from the shared buffer where used
  cx<T> ub[2][4], vv[2][4];
  const T* rin = PREP ? rec + (e / kPage) * EvLayout<K>::NITEM * kPage + (e % kPage) : nullptr;
  auto getPT = [&](int S, T* P) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if constexpr (SHARED) P[m] = __ldg(rin + (EvLayout<K>::PT + 4 * S + m) * kPage);
      else P[m] = PT[S][m];
    }
  };
  auto getQC = [&](int S, T* q) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      if constexpr (SHARED) q[c] = __ldg(rin + (EvLayout<K>::QC + 5 * S + c) * kPage);
      else q[c] = qc[S][c];
    }
  };
  if constexpr (PREP) {
    using L = EvLayout<K>;
    const T* in = rin;
    if constexpr (!SHARED) {
#pragma unroll
      for (int S = 0; S < NSUB; ++S) {
#pragma unroll
        for (int m = 0; m < 4; ++m) PT[S][m] = __ldg(in + (L::PT + 4 * S + m) * kPage);
        gprop[S] = __ldg(in + (L::GP + S) * kPage);
#pragma unroll
        for (int c = 0; c < 5; ++c) qc[S][c] = __ldg(in + (L::QC + 5 * S + c) * kPage);
      }
    }
    if constexpr (!SHARED) {
#pragma unroll
      for (int g = 0; g < K; ++g) {
        T pol[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) pol[i] = __ldg(in + (L::EPS + 5 * g + i) * kPage);
        ext_gluon(pol, (gc >> g) & 1 ? 1 : -1, g >= 2, J[g]);
      }
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
  constexpr bool kTableX = std::is_same<T, double>::value;
  cx<T> X[kTableX && !SHARED ? 2 : 1][kTableX && !SHARED ? NSEQ : 1][4];
  // SHARED: the item of sequence s for this slot's helicities: J (8 doubles), then (gamma.J) v of both
  // antitop helicities (8 each), loaded where used instead of copied to local memory
  const double* shp = SHARED ? share_event(share, e, tab->share_stride) : nullptr;
  auto sitem = [&](int s) -> const double* {
    return shp + static_cast<int64_t>(tab->share_base[s] + pext_bits(gc, tab->seq_mask[s])) * 24 * kPage;
  };
  auto ldJ = [&](int s, cx<T>* o) {   // (SHARED implies FP64)
    const double* it = sitem(s);
#pragma unroll
    for (int m = 0; m < 4; ++m) o[m] = {static_cast<T>(it[(2 * m) * kPage]), static_cast<T>(it[(2 * m + 1) * kPage])};
  };
  auto ldX = [&](int b, int s, cx<T>* o) {
    const double* it = sitem(s) + (8 + 8 * b) * kPage;
#pragma unroll
    for (int m = 0; m < 4; ++m) o[m] = {static_cast<T>(it[(2 * m) * kPage]), static_cast<T>(it[(2 * m + 1) * kPage])};
  };
  if constexpr (!SHARED)
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
      if constexpr (SHARED) {
        cx<T> jl[4], jr[4];
        T pl[4], pr[4];
        ldJ(il, jl);
        ldJ(ir, jr);
        getPT(tab->seq_mask[il], pl);
        getPT(tab->seq_mask[ir], pr);
        v3_acc(acc, jl, jr, pl, pr, rneg(rl) != rneg(rr));
      } else {
        v3_acc(acc, J[il], J[ir], PT[tab->seq_mask[il]], PT[tab->seq_mask[ir]], rneg(rl) != rneg(rr));
      }
    }
    const int n4 = tab->full_nv4[f];
    for (int k = 0; k < n4; ++k) {
      const int16_t ra = tab->full_v4[f][k][0], rb = tab->full_v4[f][k][1], rc = tab->full_v4[f][k][2];
      if constexpr (SHARED) {
        cx<T> ja[4], jb[4], jc[4];
        ldJ(rslot(ra), ja);
        ldJ(rslot(rb), jb);
        ldJ(rslot(rc), jc);
        v4_acc(acc, ja, jb, jc, gs, rneg(ra) ^ rneg(rb) ^ rneg(rc));
      } else {
        v4_acc(acc, J[rslot(ra)], J[rslot(rb)], J[rslot(rc)], gs, rneg(ra) ^ rneg(rb) ^ rneg(rc));
      }
    }
    T fz;
    if constexpr (SHARED) fz = __ldg(rin + (EvLayout<K>::GP + NSUB - 1) * kPage);
    else fz = gprop[NSUB - 1];
#pragma unroll
    for (int m = 0; m < 4; ++m) JF[f][m] = cscale(fz, acc[m]);
  }

  // ---- antitop spinors and (gamma.J) v for both antitop helicities ----
  // (gamma.J) v for every current and both antitop helicities: precomputed in FP64 (saves FP64
  // instructions); in FP32 and double-float each jamp term forms ubar-side (row spinor x gamma.J) on
  // the fly instead, keeping 2 NSEQ spinors out of the thread's local memory (FP32-pipe arithmetic is
  // cheap, memory is not).
  if constexpr (kTableX && !SHARED) {
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
  double jsum[LHE ? NCOL : 1];
  if constexpr (LHE)
    for (int c = 0; c < NCOL; ++c) jsum[c] = 0.0;
  for (int a = 0; a < 2; ++a) {
    const int h0 = hbase | (a ? bit_t : 0), h1 = h0 | bit_tb;
    const bool good0 = PER_HEL || ((mask[h0 >> 5] >> (h0 & 31)) & 1u);
    const bool good1 = PER_HEL || ((mask[h1 >> 5] >> (h1 & 31)) & 1u);
    if (!good0 && !good1) {
      if (JOUT) {
        float2* row = jout + (e * (4 << K) + slot * 4 + 2 * a) * NCOL;
        for (int c = 0; c < 2 * NCOL; ++c) row[c] = make_float2(0.f, 0.f);
      }
      if (LHE) {
        out[(slot * 4 + 2 * a) * stride + e] = 0.0;
        out[(slot * 4 + 2 * a + 1) * stride + e] = 0.0;
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
        if constexpr (SHARED) {
          if (m <= tab->pref_levels) {   // the prefix spinor from k_prefix_level
            int hm = 0;
            for (int j = 0; j < m; ++j) hm |= ((gc >> tab->perm[c][j]) & 1) << j;
            const int node = (((c / kFactorial[K - m]) << m | hm) << 1) | a;
            const double* it = shp + static_cast<int64_t>(tab->share_n * 24 + (tab->pref_off[m] + node) * 8) * kPage;
#pragma unroll
            for (int q = 0; q < 4; ++q) stk[m][q] = {it[(2 * q) * kPage], it[(2 * q + 1) * kPage]};
            continue;
          }
        }
        cx<T> acc[4] = {};
        for (int j = 0; j < m; ++j) {
          const int16_t r = tab->sub[c][j][m];
          if constexpr (SHARED) {
            cx<T> jr[4];
            ldJ(rslot(r), jr);
            row_gamma_acc(acc, stk[j], jr, rneg(r));
          } else {
            row_gamma_acc(acc, stk[j], J[rslot(r)], rneg(r));
          }
        }
        if constexpr (SHARED) {
          T q[5];
          getQC(tab->prefix_mask[c][m], q);
          row_prop(acc, q, stk[m]);
        } else {
          row_prop(acc, qc[tab->prefix_mask[c][m]], stk[m]);
        }
      }
      const int fi = tab->full_idx[c];
      const int fidx = fi >= 0 ? fi : -fi - 1;
      const bool fneg = fi < 0 && !(K & 1);   // reflection sign (-1)^(K+1)
      if constexpr (kTableX) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          cx<T> amp = mdot(Jq[b], JF[fidx]);   // all gluons on one current: ubar gamma.J v = Jq.J
          if (fneg) amp = cneg(amp);
          for (int j = 1; j < K; ++j) {
            const int16_t r = tab->sub[c][j][K];
            if constexpr (SHARED) {
              cx<T> x[4];
              ldX(b, rslot(r), x);
              sdot_acc(amp, stk[j], x, rneg(r));
            } else {
              sdot_acc(amp, stk[j], X[b][rslot(r)], rneg(r));
            }
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
        if (!good) {
          if (LHE) out[(slot * 4 + 2 * a + b) * stride + e] = 0.0;
          continue;
        }
        double v;
        if constexpr (std::is_same<T, dd::df>::value)
          v = static_cast<double>(colour_sum_hi<NCOL>(A[b], ctri)) * cst.colour_scale;
        else
          v = static_cast<double>(colour_sum<NCOL, T>(A[b], ctri)) * cst.colour_scale;
        if (PER_HEL) out[h * stride + e] = v;
        else if (LHE) out[(slot * 4 + 2 * a + b) * stride + e] = v;
        else total += v;
        if constexpr (LHE)
          for (int c = 0; c < NCOL; ++c) jsum[c] = fma(A[b][c].r, A[b][c].r, fma(A[b][c].i, A[b][c].i, jsum[c]));
      }
    }
  }
  if constexpr (LHE) {
    for (int c = 0; c < NCOL; ++c) j2[(static_cast<int64_t>(slot) * NCOL + c) * stride + e] = jsum[c];
    return;
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

// The kernel body: thread -> (event, slot) of the launch shape, then me_slot.
template <int K, class T, bool PER_HEL, bool PREP, bool JOUT, bool SHARED, bool LHE>
__device__ __forceinline__ void me_thread(const double* __restrict__ mom, const T* __restrict__ rec, int64_t nevt,
                                          const Tables* __restrict__ tab, const int* __restrict__ gslots,
                                          const int* __restrict__ nslot_dev, const uint32_t* __restrict__ mask,
                                          const typename ColourT<T>::type* __restrict__ ctri, const MeConst& cst,
                                          double* __restrict__ out, int64_t stride, float2* __restrict__ jout, int tile_ev,
                                          int slot_major, const int* __restrict__ evlist, const int* __restrict__ nlist,
                                          int rows_out, const uint8_t* __restrict__ skip, const double* __restrict__ share,
                                          double* __restrict__ j2) {
  static_assert(!SHARED || (PREP && std::is_same<T, double>::value), "shared currents: FP64 with a record");
  static_assert(!LHE || (PREP && !PER_HEL && !JOUT && std::is_same<T, double>::value), "LHE rows: FP64 with a record");
  const int tile_sl = static_cast<int>(blockDim.x) / tile_ev;   // slots per block
  const unsigned bev = slot_major ? blockIdx.y : blockIdx.x, bsl = slot_major ? blockIdx.x : blockIdx.y;
  const int64_t et = static_cast<int64_t>(bev) * tile_ev + threadIdx.x % tile_ev;
  const int slot = static_cast<int>(bsl) * tile_sl + static_cast<int>(threadIdx.x) / tile_ev;
  if (et >= nevt || slot >= *nslot_dev) return;
  // evlist: the thread works on event evlist[et] of the batch (et < *nlist), else on event et
  if (evlist && et >= *nlist) return;
  const int64_t e = evlist ? static_cast<int64_t>(evlist[et]) : et;
  if (PREP && skip && skip[e]) return;   // recomputed by another launch
  const int gc = gslots[slot];   // bit g = helicity (+1) of gluon g

  me_slot<K, T, PER_HEL, PREP, JOUT, SHARED, LHE>(mom, rec, e, slot, gc, tab, mask, ctri, cst, out, stride, jout, rows_out,
                                                share, j2);
}

template <int K, class T, bool PER_HEL, bool PREP, bool JOUT, bool SHARED = false, bool LHE = false>
__global__ void __launch_bounds__(kMeThreads)
k_me_gluonhel(const double* __restrict__ mom, const T* __restrict__ rec, int64_t nevt, const Tables* __restrict__ tab,
              const int* __restrict__ gslots, const int* __restrict__ nslot_dev, const uint32_t* __restrict__ mask,
              const typename ColourT<T>::type* __restrict__ ctri, MeConst cst, double* __restrict__ out, int64_t stride,
              float2* __restrict__ jout, int tile_ev, int slot_major, const int* __restrict__ evlist,
              const int* __restrict__ nlist, int rows_out, const uint8_t* __restrict__ skip,
              const double* __restrict__ share = nullptr, double* __restrict__ j2 = nullptr) {
  me_thread<K, T, PER_HEL, PREP, JOUT, SHARED, LHE>(mom, rec, nevt, tab, gslots, nslot_dev, mask, ctri, cst, out, stride,
                                                    jout, tile_ev, slot_major, evlist, nlist, rows_out, skip, share, j2);
}

// The FP64 slot kernel with a record, compiled for MINB resident blocks per SM: 4 for 2 and 3 gluons (at
// most 128 registers; the unbounded compile takes 168 and 166, 3 blocks), 3 for 4 and 5 (at most 168;
// unbounded 254, 2 blocks).  More warps hide more of the FP64 pipe's dependent-instruction latency:
// measured 1.3 % faster for 3 gluons, 8 % for 4 (shared currents) and 3 % for 5; spills stay below 250
// bytes per thread.  With 2 gluons it lets gg -> t tbar's 16,384 events (2,048 warps) reside in one
// wave instead of 3 blocks per SM and a tail.
template <int K, bool JOUT, bool SHARED, int MINB>
__global__ void __launch_bounds__(kMeThreads, MINB)
k_me_gluonhel_occ(const double* __restrict__ rec, int64_t nevt, const Tables* __restrict__ tab,
                 const int* __restrict__ gslots, const int* __restrict__ nslot_dev, const uint32_t* __restrict__ mask,
                 const double* __restrict__ ctri, MeConst cst, double* __restrict__ out, int64_t stride,
                 float2* __restrict__ jout, int tile_ev, int slot_major, const uint8_t* __restrict__ skip,
                 const double* __restrict__ share) {
  me_thread<K, double, false, true, JOUT, SHARED, false>(nullptr, rec, nevt, tab, gslots, nslot_dev, mask, ctri, cst, out,
                                                         stride, jout, tile_ev, slot_major, nullptr, nullptr, 0, skip,
                                                         share, nullptr);
}

// Currents shared between gluon-helicity combinations (FP64): every canonical sequence s of `level`
// gluons, for every helicity assignment h of its own gluons, from the record and the shorter sequences
// of the same assignment already in share; writes J and (gamma.J) v of both antitop helicities to item
// share_base[s] + h (the layout k_me_gluonhel<..., SHARED> reads).  One thread per (event, item of the
// level); levels run in order 1 .. K-1.
template <int K>
__global__ void __launch_bounds__(128)
k_share_level(const double* __restrict__ rec, int64_t nevt, const Tables* __restrict__ tab, MeConst cst, int level,
              int s0, int s1, double* __restrict__ share) {
  using L = EvLayout<K>;
  const int per_ev = (s1 - s0) << level;
  // thread -> (item of the level, page of 32 events, event in the page): a warp writes one item of 32
  // consecutive events, one 256-byte line per double
  const int64_t npage = (nevt + kPage - 1) / kPage;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= npage * kPage * per_ev) return;
  const int j = static_cast<int>(t / (npage * kPage));
  const int64_t e = t - j * npage * kPage;
  if (e >= nevt) return;
  const int s = s0 + (j >> level), h = j & ((1 << level) - 1);
  const int msk = tab->seq_mask[s];
  const int gc = pdep_bits(h, msk);
  const double* in = rec + (e / kPage) * L::NITEM * kPage + (e % kPage);
  auto ld = [&](int item) -> double { return __ldg(in + item * kPage); };
  double* sh = share_event(share, e, tab->share_stride);
  auto getJ = [&](int slot, cx<double>* J) {
    const double* it = sh + static_cast<int64_t>(tab->share_base[slot] + pext_bits(gc, tab->seq_mask[slot])) * 24 * kPage;
#pragma unroll
    for (int m = 0; m < 4; ++m) J[m] = {it[(2 * m) * kPage], it[(2 * m + 1) * kPage]};
  };
  auto getP = [&](int slot, double* P) {
#pragma unroll
    for (int m = 0; m < 4; ++m) P[m] = ld(L::PT + 4 * tab->seq_mask[slot] + m);
  };
  cx<double> J[4];
  if (level == 1) {
    double pol[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) pol[i] = ld(L::EPS + 5 * s + i);
    ext_gluon(pol, h ? 1 : -1, s >= 2, J);
  } else {
    const double gs = cst.gs;
    cx<double> acc[4] = {};
    const int n3 = tab->seq_nv3[s];
    for (int k = 0; k < n3; ++k) {
      const int16_t rl = tab->seq_v3[s][k][0], rr = tab->seq_v3[s][k][1];
      cx<double> JL[4], JR[4];
      double PL[4], PR[4];
      getJ(rslot(rl), JL);
      getJ(rslot(rr), JR);
      getP(rslot(rl), PL);
      getP(rslot(rr), PR);
      v3_acc(acc, JL, JR, PL, PR, rneg(rl) != rneg(rr));
    }
    const int n4 = tab->seq_nv4[s];
    for (int k = 0; k < n4; ++k) {
      const int16_t ra = tab->seq_v4[s][k][0], rb = tab->seq_v4[s][k][1], rc = tab->seq_v4[s][k][2];
      cx<double> JA[4], JB[4], JC[4];
      getJ(rslot(ra), JA);
      getJ(rslot(rb), JB);
      getJ(rslot(rc), JC);
      v4_acc(acc, JA, JB, JC, gs, rneg(ra) ^ rneg(rb) ^ rneg(rc));
    }
    const double f = ld(L::GP + msk);
#pragma unroll
    for (int m = 0; m < 4; ++m) J[m] = cscale(f, acc[m]);
  }
  double* out = sh + static_cast<int64_t>(tab->share_base[s] + h) * 24 * kPage;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    out[(2 * m) * kPage] = J[m].r;
    out[(2 * m + 1) * kPage] = J[m].i;
  }
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    cx<double> v[4], X[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = {ld(L::VV + (b * 4 + q) * 2), ld(L::VV + (b * 4 + q) * 2 + 1)};
    gamma_col(J, v, X);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      out[(8 + 8 * b + 2 * m) * kPage] = X[m].r;
      out[(8 + 8 * b + 2 * m + 1) * kPage] = X[m].i;
    }
  }
}

// Quark-line prefixes shared between gluon-helicity combinations (FP64): the row spinor after the first
// `level` gluons of an ordering, for every helicity assignment of those gluons and both top helicities,
// from the top spinor, the lower levels' nodes and the shared currents, by the same operations as the
// slot kernel's walk (so the results are bit-identical).  One thread per (event, node pair of the level):
// the two top helicities of a node share its currents' gamma.J entries and propagator coefficients.
// Levels M run in order 1 .. tab->pref_levels after the current levels (M a template argument, so that
// the per-level arrays stay in registers).
template <int K, int M>
__global__ void __launch_bounds__(128)
k_prefix_level(const double* __restrict__ rec, int64_t nevt, const Tables* __restrict__ tab,
               double* __restrict__ share) {
  using L = EvLayout<K>;
  constexpr int m = M;
  const int per_ev = (kFactorial[K] / kFactorial[K - m]) << m;   // node pairs (ordering prefix, helicities)
  // thread -> (node pair of the level, page, event in the page), as k_share_level
  const int64_t npage = (nevt + kPage - 1) / kPage;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= npage * kPage * per_ev) return;
  const int pair = static_cast<int>(t / (npage * kPage));
  const int64_t e = t - pair * npage * kPage;
  if (e >= nevt) return;
  const int h = pair & ((1 << m) - 1), p = pair >> m;
  const int c0 = p * kFactorial[K - m];   // the first ordering with this prefix
  const double* in = rec + (e / kPage) * L::NITEM * kPage + (e % kPage);
  double* sh = share_event(share, e, tab->share_stride);
  double* pref = sh + static_cast<int64_t>(tab->share_n) * 24 * kPage;
  int gcp = 0;   // the prefix gluons' helicity bits, by gluon
#pragma unroll
  for (int j = 0; j < m; ++j) gcp |= ((h >> j) & 1) << tab->perm[c0][j];
  Slash<double> g[m];
#pragma unroll
  for (int j = 0; j < m; ++j) {
    const int16_t r = tab->sub[c0][j][m];
    const double* it =
        sh + static_cast<int64_t>(tab->share_base[rslot(r)] + pext_bits(gcp, tab->seq_mask[rslot(r)])) * 24 * kPage;
    cx<double> Jr[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) Jr[q] = {it[(2 * q) * kPage], it[(2 * q + 1) * kPage]};
    g[j] = slash_of(Jr, rneg(r));
  }
  double qc[5];
  const int pm = tab->prefix_mask[c0][m];
#pragma unroll
  for (int i = 0; i < 5; ++i) qc[i] = __ldg(in + (L::QC + 5 * pm + i) * kPage);
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    cx<double> stk[m][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      stk[0][q] = {__ldg(in + (L::UB + (a * 4 + q) * 2) * kPage), __ldg(in + (L::UB + (a * 4 + q) * 2 + 1) * kPage)};
#pragma unroll
    for (int j = 1; j < m; ++j) {
      const int nj = (((c0 / kFactorial[K - j]) << j | (h & ((1 << j) - 1))) << 1) | a;
      const double* it = pref + static_cast<int64_t>(tab->pref_off[j] + nj) * 8 * kPage;
#pragma unroll
      for (int q = 0; q < 4; ++q) stk[j][q] = {it[(2 * q) * kPage], it[(2 * q + 1) * kPage]};
    }
    cx<double> acc[4] = {};
#pragma unroll
    for (int j = 0; j < m; ++j) row_slash_acc(acc, stk[j], g[j]);
    cx<double> o[4];
    row_prop(acc, qc, o);
    double* out = pref + static_cast<int64_t>(tab->pref_off[m] + (pair << 1 | a)) * 8 * kPage;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      out[(2 * q) * kPage] = o[q].r;
      out[(2 * q + 1) * kPage] = o[q].i;
    }
  }
}

}  // namespace v2
}  // namespace mg
