// mg_peak.cu -- FMA throughput microbenchmark: the ALU roofline denominators of the matrix-element
// kernels (FP64 for the plain path, FP32 for the FP32-amplitude path).  Each thread runs 8
// independent FMA chains; the grid covers every SM several times over.
#include <cuda_runtime.h>

#include "mg_alloc.h"
#include "mg_internal.h"

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_chain(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == T(12345.678)) out[0] = s;   // keeps the chains live
}

template <class T>
mg_status run(int iters, double* flops) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return MG_ECUDA;
  }
  T* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mg_status rc = MG_OK;
  if (mg::dev_alloc(&out, sizeof(T)) != cudaSuccess || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = MG_ECUDA;
  } else {
    const int blocks = nsm * 8, threads = 256;
    const T a = T(0.999999), b = T(1e-7);
    { k_fma_chain<T><<<blocks, threads, 0, st>>>(out, iters / 8 + 1, a, b); mg::note_launch(); }   // warm-up
    cudaEventRecord(e0, st);
    { k_fma_chain<T><<<blocks, threads, 0, st>>>(out, iters, a, b); mg::note_launch(); }
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = MG_ECUDA;
    } else {
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      const double n = static_cast<double>(blocks) * threads * iters * 16.0 * 8.0 * 2.0;
      *flops = n / (ms * 1e-3);
    }
  }
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (out) mg::dev_free(out);
  return rc;
}

}  // namespace

extern "C" mg_status mg_measure_fma_peak(int fp32, int iters, double* flops_per_s) {
  if (!flops_per_s || iters < 1 || iters > (1 << 20)) return MG_EINVAL;
  return fp32 ? run<float>(iters, flops_per_s) : run<double>(iters, flops_per_s);
}
