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

#include <type_traits>

#include "mg_internal.h"
#include "mg_kernels.h"
#include "mg_me_algebra.cuh"
#include "mg_me_kernel.cuh"

namespace mg {
namespace v2 {

// One thread per event: the event's record, AoSoA (page of 32 events, value-major within a page).
template <int K, class T>
__global__ void __launch_bounds__(128) k_event_prep(const double* __restrict__ mom, int64_t nevt, MeConst cst,
                                                    T* __restrict__ rec) {
  constexpr int npar = K + 2;
  using L = EvLayout<K>;
  const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (e >= nevt) return;
  double p[npar][4];
  const double* base = mom + (e / kPage) * npar * 4 * kPage + (e % kPage);
#pragma unroll
  for (int i = 0; i < npar; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) p[i][m] = __ldg(base + (i * 4 + m) * kPage);
  T* out = rec + (e / kPage) * L::NITEM * kPage + (e % kPage);
  record_all<K, T>(p, cst, [&](int i, T v) { out[i * kPage] = v; });
  if constexpr (std::is_same<T, float>::value && L::NPAIR > 0)
    record_j2<K, T>(p, cst, [&](int i, T v) { out[i * kPage] = v; });
}

// FP32 modes: events whose smallest internal invariant |P^2| or |Q^2 - m^2| (over the gluon and quark
// propagators of the recursion) is below tau * s get flag[e] = 1 and are appended to repair[] (count in
// *nrepair, zero before the launch); the others get flag[e] = 0.  FP32 rounding of the amplitudes is
// amplified ~ 1/sqrt(invariant / s) there (collinear and soft gluons).
template <int K>
__global__ void __launch_bounds__(128) k_event_flags(const double* __restrict__ mom, int64_t nevt, float mt, float tau,
                                                     int* __restrict__ repair, int* __restrict__ nrepair,
                                                     uint8_t* __restrict__ flag) {
  constexpr int npar = K + 2;
  const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (e >= nevt) return;
  double p[npar][4];
  const double* base = mom + (e / kPage) * npar * 4 * kPage + (e % kPage);
#pragma unroll
  for (int i = 0; i < npar; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) p[i][m] = __ldg(base + (i * 4 + m) * kPage);
  const bool redo = min_invariant_ratio<K>(p, mt) < tau;
  if (redo) repair[atomicAdd(nrepair, 1)] = static_cast<int>(e);
  flag[e] = redo ? 1 : 0;
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
  { v2::k_gluon_slots<<<1, 32, 0, st>>>(mask, K, gslots, n, nrows); mg::note_launch(); }
  return cudaGetLastError();
}

static int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n;
}

template <int K, class T, bool PER_HEL>
static cudaError_t launch_v2(const double* mom, void* prep, int64_t nevt, const Tables* tab, const int* gslots,
                             int maxslot, const int* nslot, const uint32_t* mask, const void* ctri_any,
                             const MeConst& cst, double* out, int64_t stride, float2* jout, MeShape shape,
                             const uint8_t* skip, const int* evlist, const int* nlist, int rows_out, cudaStream_t st,
                             const double* share) {
  const T* ctri = static_cast<const T*>(ctri_any);
  int tev = shape.tile_ev;
  if (tev != 32 && tev != 64 && tev != 128) tev = 128;
  int threads = kMeThreads;
  // a grid of fewer than 4 blocks per SM (gg -> t tbar at 16,384 events: 512 blocks of 4 warps, 3 or 4
  // per SM, one per sub-partition each): blocks of 2 warps, so that the busiest sub-partition holds
  // at most half a warp more than the average instead of a whole one
  if (prep && !PER_HEL &&
      static_cast<int64_t>((nevt + tev - 1) / tev) * ((maxslot + kMeThreads / tev - 1) / (kMeThreads / tev)) <
          4 * static_cast<int64_t>(sm_count())) {
    threads = kMeThreads / 2;
    if (tev > threads) tev = threads;
  }
  const int tsl = threads / tev;
  const unsigned nev_t = static_cast<unsigned>((nevt + tev - 1) / tev), nsl_t = static_cast<unsigned>((maxslot + tsl - 1) / tsl);
  const int sm = shape.slot_major ? 1 : 0;
  dim3 grid = sm ? dim3(nsl_t, nev_t) : dim3(nev_t, nsl_t);
  if (nev_t == 0 || nsl_t == 0) return cudaSuccess;
  if (prep && !PER_HEL) {
    const T* rec = static_cast<const T*>(prep);
    if (shape.unrolled && me_static_available(K, sizeof(T) == 4))
      return launch_me_static(K, sizeof(T) == 4, rec, nevt, gslots, maxslot, nslot, mask, cst, out, stride, jout, shape,
                              skip, st);
    if constexpr (std::is_same<T, double>::value) {
      // the compile for more resident blocks (k_me_gluonhel_occ): 2, 4 and 5 gluons, and 3 with shared
      // currents (without them its bounded compile spills ~0.5 KB per thread)
      if constexpr (K >= 2) {
        constexpr int MINB = K <= 3 ? 4 : 3;
        if (K != 3 || share) {
          if (jout && share)
            { v2::k_me_gluonhel_occ<K, true, true, MINB><<<grid, threads, 0, st>>>(
                rec, nevt, tab, gslots, nslot, mask, ctri, cst, out, stride, jout, tev, sm, skip, share); mg::note_launch(); }
          else if (share)
            { v2::k_me_gluonhel_occ<K, false, true, MINB><<<grid, threads, 0, st>>>(
                rec, nevt, tab, gslots, nslot, mask, ctri, cst, out, stride, nullptr, tev, sm, skip, share); mg::note_launch(); }
          else if (jout)
            { v2::k_me_gluonhel_occ<K, true, false, MINB><<<grid, threads, 0, st>>>(
                rec, nevt, tab, gslots, nslot, mask, ctri, cst, out, stride, jout, tev, sm, skip, nullptr); mg::note_launch(); }
          else
            { v2::k_me_gluonhel_occ<K, false, false, MINB><<<grid, threads, 0, st>>>(
                rec, nevt, tab, gslots, nslot, mask, ctri, cst, out, stride, nullptr, tev, sm, skip, nullptr); mg::note_launch(); }
          return cudaGetLastError();
        }
      }
      if (share) {
        if (jout)
          { v2::k_me_gluonhel<K, T, false, true, true, true><<<grid, threads, 0, st>>>(
              mom, rec, nevt, tab, gslots, nslot, mask, ctri, cst, out, stride, jout, tev, sm, nullptr, nullptr, 0, skip,
              share); mg::note_launch(); }
        else
          { v2::k_me_gluonhel<K, T, false, true, false, true><<<grid, threads, 0, st>>>(
              mom, rec, nevt, tab, gslots, nslot, mask, ctri, cst, out, stride, nullptr, tev, sm, nullptr, nullptr, 0,
              skip, share); mg::note_launch(); }
        return cudaGetLastError();
      }
    }
    if (jout)
      { v2::k_me_gluonhel<K, T, false, true, true><<<grid, threads, 0, st>>>(mom, rec, nevt, tab, gslots, nslot, mask,
                                                                             ctri, cst, out, stride, jout, tev, sm, nullptr,
                                                                             nullptr, 0, skip); mg::note_launch(); }
    else
      { v2::k_me_gluonhel<K, T, false, true, false><<<grid, threads, 0, st>>>(mom, rec, nevt, tab, gslots, nslot,
                                                                              mask, ctri, cst, out, stride, nullptr, tev,
                                                                              sm, nullptr, nullptr, 0, skip); mg::note_launch(); }
  } else if (PER_HEL) {
    // the helicity filter: a few thousand threads, so blocks of one warp (32 events of one slot) spread
    // them evenly over every SM; 128-thread blocks left a third of the SMs with twice the work
    const dim3 g1(static_cast<unsigned>((nevt + 31) / 32), static_cast<unsigned>(maxslot));
    { v2::k_me_gluonhel<K, T, PER_HEL, false, false><<<g1, 32, 0, st>>>(mom, nullptr, nevt, tab, gslots, nslot, mask,
                                                                       ctri, cst, out, stride, nullptr, 32, 0, evlist,
                                                                       nlist, rows_out, nullptr); mg::note_launch(); }
  } else {
    { v2::k_me_gluonhel<K, T, PER_HEL, false, false><<<grid, kMeThreads, 0, st>>>(mom, nullptr, nevt, tab, gslots, nslot,
                                                                                 mask, ctri, cst, out, stride, nullptr,
                                                                                 tev, sm, evlist, nlist, rows_out,
                                                                                 nullptr); mg::note_launch(); }
  }
  return cudaGetLastError();
}

template <int K, class T>
static cudaError_t launch_prep(const double* mom, int64_t nevt, const MeConst& cst, void* rec, cudaStream_t st) {
  if (nevt <= 0) return cudaSuccess;
  { v2::k_event_prep<K, T><<<static_cast<unsigned>((nevt + 127) / 128), 128, 0, st>>>(mom, nevt, cst, static_cast<T*>(rec)); mg::note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_event_prep(int K, bool fp32, const double* mom, int64_t nevt, const MeConst& cst, void* rec,
                              cudaStream_t st) {
  switch (K) {
    case 2: return fp32 ? launch_prep<2, float>(mom, nevt, cst, rec, st) : launch_prep<2, double>(mom, nevt, cst, rec, st);
    case 3: return fp32 ? launch_prep<3, float>(mom, nevt, cst, rec, st) : launch_prep<3, double>(mom, nevt, cst, rec, st);
    case 4: return fp32 ? launch_prep<4, float>(mom, nevt, cst, rec, st) : launch_prep<4, double>(mom, nevt, cst, rec, st);
    case 5: return fp32 ? launch_prep<5, float>(mom, nevt, cst, rec, st) : launch_prep<5, double>(mom, nevt, cst, rec, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int K>
static cudaError_t launch_share_k(const void* rec, int64_t nevt, const Tables* tab, const MeConst& cst, double* share,
                                  cudaStream_t st) {
  int s0 = 0;
  for (int level = 1; level < K; ++level) {
    int n = 1;   // canonical sequences of `level` gluons: K!/(K-level)!/2 (the K singles for level 1)
    for (int i = 0; i < level; ++i) n *= K - i;
    const int count = level == 1 ? K : n / 2;
    const int64_t threads = (nevt + kPage - 1) / kPage * kPage * (static_cast<int64_t>(count) << level);
    if (threads > 0)
      { v2::k_share_level<K><<<static_cast<unsigned>((threads + 127) / 128), 128, 0, st>>>(
          static_cast<const double*>(rec), nevt, tab, cst, level, s0, s0 + count, share); mg::note_launch(); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    s0 += count;
  }
  // then the quark-line prefixes, level by level (each reads the currents and the lower levels)
  const int levels = K - 1 < 3 ? K - 1 : 3;
  for (int m = 1; m <= levels; ++m) {
    int orderings = 1;
    for (int i = 0; i < m; ++i) orderings *= K - i;
    const int64_t threads = (nevt + kPage - 1) / kPage * kPage * (static_cast<int64_t>(orderings) << m);
    const unsigned blocks = static_cast<unsigned>((threads + 127) / 128);
    const double* r = static_cast<const double*>(rec);
    if (threads > 0) {
      if (m == 1) v2::k_prefix_level<K, 1><<<blocks, 128, 0, st>>>(r, nevt, tab, share);
      if constexpr (K >= 3) if (m == 2) v2::k_prefix_level<K, 2><<<blocks, 128, 0, st>>>(r, nevt, tab, share);
      if constexpr (K >= 4) if (m == 3) v2::k_prefix_level<K, 3><<<blocks, 128, 0, st>>>(r, nevt, tab, share);
      mg::note_launch();
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int64_t share_doubles(int K) {
  int64_t nodes = 0;
  const int levels = K - 1 < 3 ? K - 1 : 3;
  for (int m = 1; m <= levels; ++m) {
    int orderings = 1;
    for (int i = 0; i < m; ++i) orderings *= K - i;
    nodes += static_cast<int64_t>(orderings << m) * 2;
  }
  return static_cast<int64_t>(share_items(K)) * 24 + nodes * 8;
}

int share_items(int K) {
  int n = 0, total = 0;
  for (int level = 1; level < K; ++level) {
    int f = 1;
    for (int i = 0; i < level; ++i) f *= K - i;
    n = level == 1 ? K : f / 2;
    total += n << level;
  }
  return total;
}

cudaError_t launch_share(int K, const void* rec, int64_t nevt, const Tables* tab, const MeConst& cst, double* share,
                         cudaStream_t st) {
  switch (K) {
    case 2: return launch_share_k<2>(rec, nevt, tab, cst, share, st);
    case 3: return launch_share_k<3>(rec, nevt, tab, cst, share, st);
    case 4: return launch_share_k<4>(rec, nevt, tab, cst, share, st);
    case 5: return launch_share_k<5>(rec, nevt, tab, cst, share, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int K>
static cudaError_t launch_flags(const double* mom, int64_t nevt, const MeConst& cst, int* repair, int* nrepair,
                                uint8_t* flag, cudaStream_t st) {
  if (nevt <= 0) return cudaSuccess;
  { v2::k_event_flags<K><<<static_cast<unsigned>((nevt + 127) / 128), 128, 0, st>>>(
      mom, nevt, static_cast<float>(cst.mt), static_cast<float>(cst.fp32_tau), repair, nrepair, flag); mg::note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_event_flags(int K, const double* mom, int64_t nevt, const MeConst& cst, int* repair, int* nrepair,
                               uint8_t* flag, cudaStream_t st) {
  switch (K) {
    case 2: return launch_flags<2>(mom, nevt, cst, repair, nrepair, flag, st);
    case 3: return launch_flags<3>(mom, nevt, cst, repair, nrepair, flag, st);
    case 4: return launch_flags<4>(mom, nevt, cst, repair, nrepair, flag, st);
    case 5: return launch_flags<5>(mom, nevt, cst, repair, nrepair, flag, st);
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
                               const uint8_t* skip, const int* evlist, const int* nlist, int rows_out,
                               const double* share) {
#define MG_V2_CASE(KK)                                                                                              \
  case KK:                                                                                                          \
    if (per_hel) return fp32 ? launch_v2<KK, float, true>(mom, prep, nevt, tab, gslots, maxslot, nslot, mask, ctri32, cst,  \
                                                          out, stride, jout, shape, skip, evlist, nlist, rows_out, st, share)                                          \
                             : launch_v2<KK, double, true>(mom, prep, nevt, tab, gslots, maxslot, nslot, mask, ctri64, cst, \
                                                           out, stride, jout, shape, skip, evlist, nlist, rows_out, st, share);                                        \
    return fp32 ? launch_v2<KK, float, false>(mom, prep, nevt, tab, gslots, maxslot, nslot, mask, ctri32, cst, out, stride, \
                                              jout, shape, skip, evlist, nlist, rows_out, st, share)                                                                   \
                : launch_v2<KK, double, false>(mom, prep, nevt, tab, gslots, maxslot, nslot, mask, ctri64, cst, out, stride,\
                                               jout, shape, skip, evlist, nlist, rows_out, st, share);
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
