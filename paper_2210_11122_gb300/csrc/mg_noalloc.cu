// mg_noalloc.cu -- mg_sigmakin_noalloc: the FP64 matrix-element path with its scratch memory in a
// fixed, statically sized device array instead of context-owned buffers grown with cudaMalloc.
//
// Who needs this: programs that own every byte of device memory they run in -- an event generator
// embedding the engine that pre-allocates its whole GPU budget in one arena, or a host framework
// whose pooling allocator must stay the only allocator -- cannot let a library call cudaMalloc or
// cudaFree behind their back (those calls also synchronise the whole device, stalling the
// caller's other streams).  mg_sigmakin may grow its scratch on a larger batch; this entry point
// never allocates: its per-(helicity, event) partial sums live in g_noalloc_scratch below.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "mg_ctx.h"
#include "mg_internal.h"
#include "mg_kernels.h"

namespace {

// 2^21 doubles = 16 MiB, held by every GPU that loads the library until the process exits.
constexpr int64_t kScratchDoubles = int64_t(1) << 21;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Device address of g_noalloc_scratch per device.  In host code the symbol's name only stands for
// the array, so the address is fetched with cudaGetSymbolAddress, once per device, with that device
// current (the first call on each device does it).
std::mutex g_lock;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

mg_status scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return MG_ECUDA; }
  if (dev < 0 || dev >= kMaxDevices) return MG_ENOTSUP;
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MG_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return MG_OK;
}

int64_t pad_page(int64_t n) { return (n + mg::kPage - 1) / mg::kPage * mg::kPage; }

}  // namespace

extern "C" mg_status mg_sigmakin_noalloc(mg_ctx* ctx, const double* mom_dev, int64_t nevt, double* me_dev,
                                         void* stream) {
  if (!ctx || nevt < 0 || (nevt > 0 && (!mom_dev || !me_dev))) return MG_EINVAL;
  if (!ctx->mask_ready) return MG_EINVAL;                      // needs a helicity mask (mg_hel_filter)
  if (nevt == 0) return MG_OK;
  const int64_t stride = pad_page(nevt);
  if (stride > kScratchDoubles / ctx->nhel) return MG_EINVAL;  // beyond the fixed scratch: split the batch
  double* scratch = nullptr;
  mg_status s = scratch_for_current_device(&scratch);
  if (s != MG_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ctx->last = st;
  mg::MeConst cst;
  cst.gs = std::sqrt(4.0 * 3.14159265358979323846 * ctx->prm.alphas);
  cst.mt = ctx->prm.mt;
  cst.wt = ctx->prm.wt;
  cst.colour_scale = cst.gs * cst.gs / static_cast<double>(ctx->colour_den);
  const double norm = 1.0 / (256.0 * mg::factorial(ctx->ng));
  // every element the sum kernel reads (good slots x events) is written first: nothing to clear
  if (ctx->prm.wt == 0.0) {
    if (mg::launch_me_gluonhel(ctx->K, false, false, mom_dev, nullptr, nevt, ctx->d_tab, ctx->d_gslots, 1 << ctx->K,
                               ctx->d_ngslots, ctx->d_mask, ctx->d_ctri, ctx->d_ctri_f, cst, scratch, stride, st) != cudaSuccess)
      return MG_ECUDA;
    if (mg::launch_hel_sum(scratch, ctx->d_ngslots, nevt, stride, norm, me_dev, st) != cudaSuccess) return MG_ECUDA;
  } else {
    if (mg::launch_me_helicity(ctx->K, false, mom_dev, nevt, ctx->d_tab, ctx->d_good, ctx->nhel, ctx->d_ngood,
                               ctx->d_ctri, cst, scratch, stride, st) != cudaSuccess)
      return MG_ECUDA;
    if (mg::launch_hel_sum(scratch, ctx->d_ngood, nevt, stride, norm, me_dev, st) != cudaSuccess) return MG_ECUDA;
  }
  return MG_OK;
}
