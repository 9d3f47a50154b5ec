// mg_me3_k4f.cu -- the compile-time-unrolled FP32 matrix-element kernel of mg_me3.cuh for K = 4 gluons,
// per-event record computed in the kernel.
#include "mg_me3.cuh"

namespace mg {

cudaError_t me3_upload_k4f(int K, const double* tri, int n) { return me3_upload_tu(K, tri, n); }

cudaError_t me3_fused_k4(const double* mom, int64_t nevt, const int* gslots, const int* nslot, const uint32_t* mask,
                         const MeConst& cst, double* out, int64_t stride, float2* jout, const uint8_t* skip,
                         cudaStream_t st) {
  return launch_fused<4, float>(mom, nevt, gslots, nslot, mask, cst, out, stride, jout, skip, st);
}

}  // namespace mg
