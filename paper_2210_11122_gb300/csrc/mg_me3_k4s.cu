// mg_me3_k4s.cu -- the compile-time-unrolled FP32 matrix-element kernel of mg_me3.cuh for K = 4 gluons,
// per-event record read from global memory.
#include "mg_me3.cuh"

namespace mg {

cudaError_t me3_upload_k4s(int K, const double* tri, int n) { return me3_upload_tu(K, tri, n); }

cudaError_t me3_static_k4(const void* rec, int64_t nevt, const int* gslots, int maxslot, const int* nslot,
                          const uint32_t* mask, const MeConst& cst, double* out, int64_t stride, float2* jout,
                          MeShape shape, const uint8_t* skip, cudaStream_t st) {
  return launch_static<4, float>(rec, nevt, gslots, maxslot, nslot, mask, cst, out, stride, jout, shape, skip, st);
}

}  // namespace mg
