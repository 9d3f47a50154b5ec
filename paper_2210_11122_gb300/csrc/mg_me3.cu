// mg_me3.cu -- dispatch of the matrix-element kernels with the recursion expanded at compile time
// (mg_me3.cuh; instantiated in mg_me3_k23.cu, mg_me3_k4s.cu and mg_me3_k4f.cu): availability, the
// per-device upload of their constant-memory colour triangles, and the launch entry points.
#include <cuda_runtime.h>

#include <mutex>

#include "mg_internal.h"
#include "mg_kernels.h"

namespace mg {

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

namespace {
std::mutex g_tri_mu;
bool g_tri_done[64][6] = {};
constexpr int kTriLen[6] = {0, 0, 3, 21, 300, 0};   // packed upper triangles for K = 2, 3, 4
}  // namespace

bool me_static_available(int K, bool fp32) { return fp32 && K >= 2 && K <= 4; }

cudaError_t me_static_upload_colour(int K, const double* tri, int n) {
  if (K < 2 || K > 4) return cudaSuccess;
  if (n != kTriLen[K]) return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_tri_mu);
  if (g_tri_done[dev][K]) return cudaSuccess;
  e = K < 4 ? me3_upload_k23(K, tri, n) : me3_upload_k4s(K, tri, n);
  if (e == cudaSuccess && K == 4) e = me3_upload_k4f(K, tri, n);
  if (e == cudaSuccess) g_tri_done[dev][K] = true;
  return e;
}

cudaError_t launch_me_fused(int K, bool fp32, const double* mom, int64_t nevt, const int* gslots, const int* nslot,
                            const uint32_t* mask, const MeConst& cst, double* out, int64_t stride, float2* jout,
                            const uint8_t* skip, cudaStream_t st) {
  if (!me_static_available(K, fp32)) return cudaErrorInvalidValue;
  if (K == 4) return me3_fused_k4(mom, nevt, gslots, nslot, mask, cst, out, stride, jout, skip, st);
  return me3_fused_k23(K, mom, nevt, gslots, nslot, mask, cst, out, stride, jout, skip, st);
}

cudaError_t launch_me_static(int K, bool fp32, const void* rec, int64_t nevt, const int* gslots, int maxslot,
                             const int* nslot, const uint32_t* mask, const MeConst& cst, double* out, int64_t stride,
                             float2* jout, MeShape shape, const uint8_t* skip, cudaStream_t st) {
  if (!me_static_available(K, fp32)) return cudaErrorInvalidValue;
  if (K == 4) return me3_static_k4(rec, nevt, gslots, maxslot, nslot, mask, cst, out, stride, jout, shape, skip, st);
  return me3_static_k23(K, rec, nevt, gslots, maxslot, nslot, mask, cst, out, stride, jout, shape, skip, st);
}

}  // namespace mg
