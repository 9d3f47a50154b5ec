// mg_me_dd.cu -- the FP32 modes' recomputation of the events with a small internal invariant
// (launch_me_repair): the run-time-table matrix-element kernel of mg_me_kernel.cuh with double-float
// amplitudes (~48 bits carried on the FP32 pipe, ~1/4 of the FP64 pipe's cost on GB300, where FP64
// runs at 1/64 of the FP32 rate), per-event data computed in FP64, colour sums in FP32.
#include <cuda_runtime.h>

#include "mg_internal.h"
#include "mg_kernels.h"
#include "mg_me_kernel.cuh"

namespace mg {

template <int K>
static cudaError_t launch_dd(const double* mom, int64_t nevt, const Tables* tab, const int* gslots, int maxslot,
                             const int* nslot, const uint32_t* mask, const float* ctri32, const MeConst& cst,
                             double* out, int64_t stride, const int* evlist, const int* nlist, int rows_out,
                             cudaStream_t st) {
  constexpr int tev = 128;
  const int tsl = kMeThreads / tev;
  const unsigned nev_t = static_cast<unsigned>((nevt + tev - 1) / tev), nsl_t = static_cast<unsigned>((maxslot + tsl - 1) / tsl);
  if (nev_t == 0 || nsl_t == 0) return cudaSuccess;
  { v2::k_me_gluonhel<K, dd::df, false, false, false><<<dim3(nev_t, nsl_t), kMeThreads, 0, st>>>(
      mom, nullptr, nevt, tab, gslots, nslot, mask, ctri32, cst, out, stride, nullptr, tev, 0, evlist, nlist, rows_out,
      nullptr); mg::note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_me_repair(int K, const double* mom, int64_t nevt, const Tables* tab, const int* gslots, int maxslot,
                             const int* nslot, const uint32_t* mask, const float* ctri32, const float* cfull,
                             const MeConst& cst, double* out, int64_t stride, const int* evlist, const int* nlist,
                             int rows_out, cudaStream_t st) {
  // 4 and 5 gluons: a group of lanes per (event, slot), the state in shared memory (the per-thread form
  // keeps ~28 KB of double-float arrays per thread in local memory and runs as one long wave)
  if (K >= 4)
    return launch_me_warp_repair(K, mom, nevt, tab, gslots, maxslot, nslot, mask, cfull, cst, out, stride, evlist, nlist,
                                 rows_out, st);
  switch (K) {
    case 2: return launch_dd<2>(mom, nevt, tab, gslots, maxslot, nslot, mask, ctri32, cst, out, stride, evlist, nlist, rows_out, st);
    case 3: return launch_dd<3>(mom, nevt, tab, gslots, maxslot, nslot, mask, ctri32, cst, out, stride, evlist, nlist, rows_out, st);
    case 4: return launch_dd<4>(mom, nevt, tab, gslots, maxslot, nslot, mask, ctri32, cst, out, stride, evlist, nlist, rows_out, st);
    case 5: return launch_dd<5>(mom, nevt, tab, gslots, maxslot, nslot, mask, ctri32, cst, out, stride, evlist, nlist, rows_out, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mg
