// mg_me3.cuh -- matrix-element kernel with the recursion expanded at compile time.
//
// Same thread mapping, record input and output as k_me_gluonhel of mg_me2.cu (one thread per (event,
// gluon-helicity combination), the 4 top/antitop helicity pairs in the thread, per-event record from
// k_event_prep), but the Berends-Giele recursion (mg_static_tables.h) is unrolled into straight-line
// code: every current and every prefix spinor has a fixed name, so the thread's current arrays live in
// registers (mg_me2.cu indexes them from run-time tables, which puts them in local memory); the signs of
// the reflection identity fold into the FMA operands; and the colour matrix sits in constant memory,
// read as an FMA operand.  Used where its registers fit: FP32 amplitudes for K <= 4 gluons.
//
// The kernels are instantiated in three translation units (mg_me3_k23.cu: K = 2, 3; mg_me3_k4s.cu and
// mg_me3_k4f.cu: K = 4 with the record read from global memory or computed in the kernel), which compile
// in parallel; each unit holds its own constant-memory copy of the colour triangles, filled by its
// me3_upload_* function.
#ifndef MG_ME3_CUH
#define MG_ME3_CUH
#include <cuda_runtime.h>

#include <mutex>

#include "mg_internal.h"
#include "mg_kernels.h"
#include "mg_me_algebra.cuh"
#include "mg_static_tables.h"

namespace mg {
namespace st {

static_assert(nseq<3>() == 6 && nfull<3>() == 3 && ncol<3>() == 6, "recursion tables, K = 3");
static_assert(nseq<4>() == 22 && nfull<4>() == 12 && ncol<4>() == 24, "recursion tables, K = 4");
static_assert(nseq<5>() == 105 && nfull<5>() == 60 && ncol<5>() == 120, "recursion tables, K = 5");

template <int N> struct IC { static constexpr int value = N; };

template <int B, int E, class F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (B < E) {
    f(IC<B>());
    sfor<B + 1, E>(f);
  }
}

// packed upper triangles of the colour matrices (off-diagonal entries doubled) for K = 2, 3, 4
constexpr int kTriOff[6] = {0, 0, 0, 3, 24, 324};
static __constant__ float c_tri_f[324];
static __constant__ double c_tri_d[324];

template <class T> __device__ __forceinline__ T tri(int i);
template <> __device__ __forceinline__ float tri<float>(int i) { return c_tri_f[i]; }
template <> __device__ __forceinline__ double tri<double>(int i) { return c_tri_d[i]; }

using v2::cx;

// The matrix element of event e for gluon-helicity slot `slot` (gluon helicities gc), its record read
// through ld(item): out[slot * stride + e] = sum over the slot's good helicities of the colour sums, or
// (JOUT) the jamps of its four helicities into jout.
template <int K, class T, bool JOUT, class Ld>
__device__ __forceinline__ void me_static_body(Ld&& ld, int64_t e, int slot, int gc, const uint32_t* __restrict__ mask,
                                               const MeConst& cst, double* __restrict__ out, int64_t stride,
                                               float2* __restrict__ jout) {
  constexpr int npar = K + 2;
  using L = v2::EvLayout<K>;
  constexpr int NSEQ = nseq<K>();
  constexpr int NCOL = ncol<K>();
  constexpr int NFULL = nfull<K>();
  constexpr int NSUB = 1 << K;
  constexpr int TRI = kTriOff[K];
  const T gs = static_cast<T>(cst.gs);

  // ---- gluon currents: external polarisations, then every canonical sequence by length ----
  cx<T> J[NSEQ][4];
  sfor<0, K>([&](auto gI) {
    constexpr int g = decltype(gI)::value;
    T pol[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) pol[i] = ld(L::EPS + 5 * g + i);
    v2::ext_gluon(pol, (gc >> g) & 1 ? 1 : -1, g >= 2, J[g]);
  });
  sfor<K, NSEQ>([&](auto sI) {
    constexpr int s = decltype(sI)::value;
    cx<T> acc[4] = {};
    sfor<0, nv3<K>(s)>([&](auto kI) {
      constexpr int k = decltype(kI)::value;
      constexpr int rl = v3<K>(s, k, 0), rr = v3<K>(s, k, 1);
      T PL[4], PR[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        PL[m] = ld(L::PT + 4 * smask<K>(rl >> 1) + m);
        PR[m] = ld(L::PT + 4 * smask<K>(rr >> 1) + m);
      }
      v2::v3_acc(acc, J[rl >> 1], J[rr >> 1], PL, PR, ((rl ^ rr) & 1) != 0);
    });
    sfor<0, nv4<K>(s)>([&](auto kI) {
      constexpr int k = decltype(kI)::value;
      constexpr int ra = v4<K>(s, k, 0), rb = v4<K>(s, k, 1), rc = v4<K>(s, k, 2);
      v2::v4_acc(acc, J[ra >> 1], J[rb >> 1], J[rc >> 1], gs, ((ra ^ rb ^ rc) & 1) != 0);
    });
    const T f = ld(L::GP + smask<K>(s));
#pragma unroll
    for (int m = 0; m < 4; ++m) J[s][m] = v2::cscale(f, acc[m]);
  });
  // all gluons on one current (canonical orderings)
  cx<T> JF[NFULL][4];
  {
    const T fz = ld(L::GP + NSUB - 1);
    sfor<0, NFULL>([&](auto fI) {
      constexpr int f = decltype(fI)::value;
      cx<T> acc[4] = {};
      sfor<0, fnv3<K>(f)>([&](auto kI) {
        constexpr int k = decltype(kI)::value;
        constexpr int rl = fv3<K>(f, k, 0), rr = fv3<K>(f, k, 1);
        T PL[4], PR[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          PL[m] = ld(L::PT + 4 * smask<K>(rl >> 1) + m);
          PR[m] = ld(L::PT + 4 * smask<K>(rr >> 1) + m);
        }
        v2::v3_acc(acc, J[rl >> 1], J[rr >> 1], PL, PR, ((rl ^ rr) & 1) != 0);
      });
      sfor<0, fnv4<K>(f)>([&](auto kI) {
        constexpr int k = decltype(kI)::value;
        constexpr int ra = fv4<K>(f, k, 0), rb = fv4<K>(f, k, 1), rc = fv4<K>(f, k, 2);
        v2::v4_acc(acc, J[ra >> 1], J[rb >> 1], J[rc >> 1], gs, ((ra ^ rb ^ rc) & 1) != 0);
      });
#pragma unroll
      for (int m = 0; m < 4; ++m) JF[f][m] = v2::cscale(fz, acc[m]);
    });
  }

  // helicity index of (gc, top helicity a, antitop helicity b)
  int hbase = 0;
#pragma unroll
  for (int g = 0; g < K; ++g)
    if ((gc >> g) & 1) hbase |= 1 << (npar - 1 - (g < 2 ? g : g + 2));
  const int bit_t = 1 << (npar - 3), bit_tb = 1 << (npar - 4);

  cx<T> vv[2][4];
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int q = 0; q < 4; ++q) vv[b][q] = {ld(L::VV + (b * 4 + q) * 2), ld(L::VV + (b * 4 + q) * 2 + 1)};

  double total = 0.0;
#pragma unroll 1
  for (int a = 0; a < 2; ++a) {
    const int h0 = hbase | (a ? bit_t : 0), h1 = h0 | bit_tb;
    const bool good0 = (mask[h0 >> 5] >> (h0 & 31)) & 1u;
    const bool good1 = (mask[h1 >> 5] >> (h1 & 31)) & 1u;
    if (!good0 && !good1) {
      if (JOUT) {
        float2* row = jout + (e * (4 << K) + slot * 4 + 2 * a) * NCOL;
        for (int c = 0; c < 2 * NCOL; ++c) row[c] = make_float2(0.f, 0.f);
      }
      continue;
    }
    // quark line: ubar of the top, then one prefix spinor per leading part of the ordering
    cx<T> stk[K][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) stk[0][q] = {ld(L::UB + (a * 4 + q) * 2), ld(L::UB + (a * 4 + q) * 2 + 1)};
    cx<T> Jq[2][4];
    v2::quark_current(stk[0], vv[0], Jq[0]);
    v2::quark_current(stk[0], vv[1], Jq[1]);
    cx<T> A[2][NCOL];
    sfor<0, NCOL>([&](auto cI) {
      constexpr int c = decltype(cI)::value;
      sfor<lcp<K>(c) + 1, K>([&](auto mI) {
        constexpr int m = decltype(mI)::value;
        cx<T> acc[4] = {};
        sfor<0, m>([&](auto jI) {
          constexpr int j = decltype(jI)::value;
          constexpr int r = sub<K>(c, j, m);
          v2::row_gamma_acc(acc, stk[j], J[r >> 1], (r & 1) != 0);
        });
        T q[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) q[k] = ld(L::QC + 5 * pmask<K>(c, m) + k);
        v2::row_prop(acc, q, stk[m]);
      });
      constexpr int fi = fidx<K>(c);
      constexpr int fj = fi >= 0 ? fi : -fi - 1;
      constexpr bool fneg = fi < 0 && !(K & 1);   // reflection sign (-1)^(K+1)
      cx<T> amp0 = v2::mdot(Jq[0], JF[fj]), amp1 = v2::mdot(Jq[1], JF[fj]);
      if (fneg) {
        amp0 = v2::cneg(amp0);
        amp1 = v2::cneg(amp1);
      }
      sfor<1, K>([&](auto jI) {
        constexpr int j = decltype(jI)::value;
        constexpr int r = sub<K>(c, j, K);
        cx<T> t[4] = {};
        v2::row_gamma_acc(t, stk[j], J[r >> 1], (r & 1) != 0);
        v2::sdot_acc(amp0, t, vv[0], false);
        v2::sdot_acc(amp1, t, vv[1], false);
      });
      A[0][c] = amp0;
      A[1][c] = amp1;
    });
    if constexpr (JOUT) {
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const bool good = b ? good1 : good0;
        float2* row = jout + (e * (4 << K) + slot * 4 + 2 * a + b) * NCOL;
#pragma unroll
        for (int c = 0; c < NCOL; ++c)
          row[c] = good ? make_float2(static_cast<float>(A[b][c].r), static_cast<float>(A[b][c].i))
                        : make_float2(0.f, 0.f);
      }
    } else {
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        if (!(b ? good1 : good0)) continue;
        T sum = 0;
#pragma unroll
        for (int x = 0; x < NCOL; ++x) {
          T wr = 0, wi = 0;
#pragma unroll
          for (int y = x; y < NCOL; ++y) {
            const T cxy = tri<T>(TRI + x * NCOL - x * (x - 1) / 2 + (y - x));
            wr = fma(cxy, A[b][y].r, wr);
            wi = fma(cxy, A[b][y].i, wi);
          }
          sum = fma(A[b][x].r, wr, sum);
          sum = fma(A[b][x].i, wi, sum);
        }
        total += static_cast<double>(sum) * cst.colour_scale;
      }
    }
  }
  if (!JOUT) out[slot * stride + e] = total;
}

// Record from the per-event kernel (global memory); one thread per (event, slot), launch shape as mg_me2.cu.
template <int K, class T, bool JOUT>
__global__ void __launch_bounds__(kMeThreads)
k_me_static(const T* __restrict__ rec, int64_t nevt, const int* __restrict__ gslots, const int* __restrict__ nslot_dev,
            const uint32_t* __restrict__ mask, MeConst cst, double* __restrict__ out, int64_t stride,
            float2* __restrict__ jout, int tile_ev, int slot_major, const uint8_t* __restrict__ skip) {
  using L = v2::EvLayout<K>;
  const int tile_sl = kMeThreads / tile_ev;
  const unsigned bev = slot_major ? blockIdx.y : blockIdx.x, bsl = slot_major ? blockIdx.x : blockIdx.y;
  const int64_t e = static_cast<int64_t>(bev) * tile_ev + threadIdx.x % tile_ev;
  const int slot = static_cast<int>(bsl) * tile_sl + static_cast<int>(threadIdx.x) / tile_ev;
  if (e >= nevt || slot >= *nslot_dev) return;
  if (skip && skip[e]) return;   // recomputed by another launch
  const T* in = rec + (e / kPage) * L::NITEM * kPage + (e % kPage);
  me_static_body<K, T, JOUT>([&](int item) -> T { return __ldg(in + item * kPage); }, e, slot, gslots[slot], mask, cst,
                             out, stride, jout);
}

// Record computed in the kernel: a block takes 32 events (one per lane); its four warps first compute the
// four parts of their records in FP64 (subsets of the lower and upper half, gluon polarisations, top
// spinors) into shared memory, then each warp runs the matrix elements of slots warp, warp + 4, ... of
// the 32 events.  The FP64 record work of one block overlaps the FP32 work of the others on the SM.
template <int K, class T, bool JOUT>
__global__ void __launch_bounds__(kMeThreads)
k_me_fused(const double* __restrict__ mom, int64_t nevt, const int* __restrict__ gslots, const int* __restrict__ nslot_dev,
           const uint32_t* __restrict__ mask, MeConst cst, double* __restrict__ out, int64_t stride,
           float2* __restrict__ jout, const uint8_t* __restrict__ skip) {
  static_assert(kMeThreads == 128, "four warps: four record parts");
  using L = v2::EvLayout<K>;
  constexpr int npar = K + 2, NSUB = 1 << K;
  __shared__ T rec[L::NBASE * 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * 32 + lane;
  if (e < nevt) {
    double p[npar][4];
    const double* base = mom + (e / kPage) * npar * 4 * kPage + (e % kPage);
#pragma unroll
    for (int i = 0; i < npar; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) p[i][m] = __ldg(base + (i * 4 + m) * kPage);
    auto put = [&](int i, T v) { rec[i * 32 + lane] = v; };
    if (warp == 0) v2::record_subsets<K, T, 0, NSUB / 2>(p, cst, put);
    else if (warp == 1) v2::record_subsets<K, T, NSUB / 2, NSUB>(p, cst, put);
    else if (warp == 2) v2::record_pols<K, T>(p, put);
    else v2::record_tops<K, T>(p, cst, put);
  }
  __syncthreads();
  if (e >= nevt || (skip && skip[e])) return;   // skipped events: recomputed by another launch
  const int nslot = *nslot_dev;
  for (int slot = warp; slot < nslot; slot += 4)
    me_static_body<K, T, JOUT>([&](int item) -> T { return rec[item * 32 + lane]; }, e, slot, gslots[slot], mask, cst,
                               out, stride, jout);
}

}  // namespace st

// the colour triangle of K gluons into this translation unit's constant memory (current device)
static inline cudaError_t me3_upload_tu(int K, const double* tri, int n) {
  float f[324];
  for (int i = 0; i < n; ++i) f[i] = static_cast<float>(tri[i]);
  const size_t off = static_cast<size_t>(st::kTriOff[K]);
  cudaError_t e = cudaMemcpyToSymbol(st::c_tri_d, tri, n * sizeof(double), off * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(st::c_tri_f, f, n * sizeof(float), off * sizeof(float));
  return e;
}

template <int K, class T>
static inline cudaError_t launch_static(const void* rec, int64_t nevt, const int* gslots, int maxslot, const int* nslot,
                                 const uint32_t* mask, const MeConst& cst, double* out, int64_t stride, float2* jout,
                                 MeShape shape, const uint8_t* skip, cudaStream_t stream) {
  int tev = shape.tile_ev;
  if (tev != 32 && tev != 64 && tev != 128) tev = 128;
  const int tsl = kMeThreads / tev;
  const unsigned nev_t = static_cast<unsigned>((nevt + tev - 1) / tev), nsl_t = static_cast<unsigned>((maxslot + tsl - 1) / tsl);
  if (nev_t == 0 || nsl_t == 0) return cudaSuccess;
  const int sm = shape.slot_major ? 1 : 0;
  const dim3 grid = sm ? dim3(nsl_t, nev_t) : dim3(nev_t, nsl_t);
  const T* r = static_cast<const T*>(rec);
  if (jout)
    { st::k_me_static<K, T, true><<<grid, kMeThreads, 0, stream>>>(r, nevt, gslots, nslot, mask, cst, out, stride, jout,
                                                                 tev, sm, skip); mg::note_launch(); }
  else
    { st::k_me_static<K, T, false><<<grid, kMeThreads, 0, stream>>>(r, nevt, gslots, nslot, mask, cst, out, stride,
                                                                  nullptr, tev, sm, skip); mg::note_launch(); }
  return cudaGetLastError();
}

template <int K, class T>
static inline cudaError_t launch_fused(const double* mom, int64_t nevt, const int* gslots, const int* nslot,
                                const uint32_t* mask, const MeConst& cst, double* out, int64_t stride, float2* jout,
                                const uint8_t* skip, cudaStream_t stream) {
  const unsigned blocks = static_cast<unsigned>((nevt + 31) / 32);
  if (blocks == 0) return cudaSuccess;
  if (jout)
    { st::k_me_fused<K, T, true><<<blocks, kMeThreads, 0, stream>>>(mom, nevt, gslots, nslot, mask, cst, out, stride, jout,
                                                                  skip); mg::note_launch(); }
  else
    { st::k_me_fused<K, T, false><<<blocks, kMeThreads, 0, stream>>>(mom, nevt, gslots, nslot, mask, cst, out, stride,
                                                                   nullptr, skip); mg::note_launch(); }
  return cudaGetLastError();
}

// per-unit entry points (defined in mg_me3_k23.cu, mg_me3_k4s.cu, mg_me3_k4f.cu)
cudaError_t me3_upload_k23(int K, const double* tri, int n);
cudaError_t me3_upload_k4s(int K, const double* tri, int n);
cudaError_t me3_upload_k4f(int K, const double* tri, int n);
cudaError_t me3_static_k23(int K, const void* rec, int64_t nevt, const int* gslots, int maxslot, const int* nslot,
                           const uint32_t* mask, const MeConst& cst, double* out, int64_t stride, float2* jout,
                           MeShape shape, const uint8_t* skip, cudaStream_t st);
cudaError_t me3_static_k4(const void* rec, int64_t nevt, const int* gslots, int maxslot, const int* nslot,
                          const uint32_t* mask, const MeConst& cst, double* out, int64_t stride, float2* jout,
                          MeShape shape, const uint8_t* skip, cudaStream_t st);
cudaError_t me3_fused_k23(int K, const double* mom, int64_t nevt, const int* gslots, const int* nslot,
                          const uint32_t* mask, const MeConst& cst, double* out, int64_t stride, float2* jout,
                          const uint8_t* skip, cudaStream_t st);
cudaError_t me3_fused_k4(const double* mom, int64_t nevt, const int* gslots, const int* nslot, const uint32_t* mask,
                         const MeConst& cst, double* out, int64_t stride, float2* jout, const uint8_t* skip,
                         cudaStream_t st);

}  // namespace mg

#endif  // MG_ME3_CUH
