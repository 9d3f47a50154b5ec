// mg_me3_k23.cu -- the compile-time-unrolled FP32 matrix-element kernels of mg_me3.cuh for K = 2 and 3
// gluons (record from global memory, or computed in the kernel).
#include "mg_me3.cuh"

namespace mg {

cudaError_t me3_upload_k23(int K, const double* tri, int n) { return me3_upload_tu(K, tri, n); }

cudaError_t me3_static_k23(int K, const void* rec, int64_t nevt, const int* gslots, int maxslot, const int* nslot,
                           const uint32_t* mask, const MeConst& cst, double* out, int64_t stride, float2* jout,
                           MeShape shape, const uint8_t* skip, cudaStream_t st) {
  if (K == 2) return launch_static<2, float>(rec, nevt, gslots, maxslot, nslot, mask, cst, out, stride, jout, shape, skip, st);
  if (K == 3) return launch_static<3, float>(rec, nevt, gslots, maxslot, nslot, mask, cst, out, stride, jout, shape, skip, st);
  return cudaErrorInvalidValue;
}

cudaError_t me3_fused_k23(int K, const double* mom, int64_t nevt, const int* gslots, const int* nslot,
                          const uint32_t* mask, const MeConst& cst, double* out, int64_t stride, float2* jout,
                          const uint8_t* skip, cudaStream_t st) {
  if (K == 2) return launch_fused<2, float>(mom, nevt, gslots, nslot, mask, cst, out, stride, jout, skip, st);
  if (K == 3) return launch_fused<3, float>(mom, nevt, gslots, nslot, mask, cst, out, stride, jout, skip, st);
  return cudaErrorInvalidValue;
}

}  // namespace mg
