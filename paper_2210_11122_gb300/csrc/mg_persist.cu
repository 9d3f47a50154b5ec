// mg_persist.cu -- the FP64 matrix elements of several jobs (any mix of the four processes) in ONE
// persistent kernel launch.
//
// The paper (Sec. 4) finds the GPU throughput still growing up to batches of ~16k events: smaller batches
// leave the device underfilled.  A batch of many small jobs therefore runs better as one launch whose
// thread blocks drain a common queue of work tiles than as one launch per job.  Here the queue holds
// (job, gluon-helicity slot, 128-event tile) triples, the jobs ordered by falling cost per tile (more
// gluons first, so the longest tiles start first); each 128-thread block takes the next tile from an
// atomic counter until the queue is empty, and runs the same per-thread FP64 work as k_me_gluonhel (the
// per-event record from k_event_prep; the currents and quark-line prefixes shared between a job's
// gluon-helicity combinations from its k_share_level / k_prefix_level passes where its context's FP64
// shape shares them and the job's buffer fits 2 GiB, else built in the thread).  The results are
// bit-identical to mg_sigmakin(MG_FP64), with or without the shared currents.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mg_alloc.h"
#include "mg_ctx.h"
#include "mg_internal.h"
#include "mg_kernels.h"
#include "mg_me_kernel.cuh"

namespace mg {
namespace pers {

constexpr int kMaxJobs = 64;   // the job table travels as the kernel's parameter (8 KB)
constexpr int kTileEv = 128;

struct PJob {
  const double* rec;        // per-event FP64 record
  const Tables* tab;
  const int* gslots;        // gluon-helicity combinations with a good helicity
  const int* nslot;
  const uint32_t* mask;
  const double* ctri;
  const double* share;      // the job's shared currents and prefixes (k_share_level), or null: none
  double* part;             // part[slot * stride + e]
  int64_t nevt, stride, tile0;
  int K, ntile_ev;
  MeConst cst;
};

struct PBatch {
  int njobs;
  int64_t ntiles;
  PJob job[kMaxJobs];
};

__global__ void __launch_bounds__(kMeThreads, 3) k_me_persistent(const __grid_constant__ PBatch b,
                                                              unsigned long long* __restrict__ next) {
  __shared__ long long s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = static_cast<long long>(atomicAdd(next, 1ull));
    __syncthreads();
    const int64_t tile = s_tile;
    __syncthreads();
    if (tile >= b.ntiles) return;
    int lo = 0, hi = b.njobs - 1;   // the job holding the tile: the last one with tile0 <= tile
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (b.job[mid].tile0 <= tile) lo = mid;
      else hi = mid - 1;
    }
    const PJob& J = b.job[lo];
    const int64_t t = tile - J.tile0;
    const int slot = static_cast<int>(t / J.ntile_ev);
    const int64_t e = (t - static_cast<int64_t>(slot) * J.ntile_ev) * kTileEv + threadIdx.x;
    if (e >= J.nevt || slot >= *J.nslot) continue;
    const int gc = J.gslots[slot];
    if (J.share) {
      switch (J.K) {
        case 2:
          v2::me_slot<2, double, false, true, false, true>(nullptr, J.rec, e, slot, gc, J.tab, J.mask, J.ctri, J.cst,
                                                           J.part, J.stride, nullptr, 0, J.share, nullptr);
          break;
        case 3:
          v2::me_slot<3, double, false, true, false, true>(nullptr, J.rec, e, slot, gc, J.tab, J.mask, J.ctri, J.cst,
                                                           J.part, J.stride, nullptr, 0, J.share, nullptr);
          break;
        case 4:
          v2::me_slot<4, double, false, true, false, true>(nullptr, J.rec, e, slot, gc, J.tab, J.mask, J.ctri, J.cst,
                                                           J.part, J.stride, nullptr, 0, J.share, nullptr);
          break;
        default:
          v2::me_slot<5, double, false, true, false, true>(nullptr, J.rec, e, slot, gc, J.tab, J.mask, J.ctri, J.cst,
                                                           J.part, J.stride, nullptr, 0, J.share, nullptr);
          break;
      }
      continue;
    }
    switch (J.K) {
      case 2:
        v2::me_slot<2, double, false, true, false>(nullptr, J.rec, e, slot, gc, J.tab, J.mask, J.ctri, J.cst, J.part,
                                                   J.stride, nullptr, 0, nullptr, nullptr);
        break;
      case 3:
        v2::me_slot<3, double, false, true, false>(nullptr, J.rec, e, slot, gc, J.tab, J.mask, J.ctri, J.cst, J.part,
                                                   J.stride, nullptr, 0, nullptr, nullptr);
        break;
      case 4:
        v2::me_slot<4, double, false, true, false>(nullptr, J.rec, e, slot, gc, J.tab, J.mask, J.ctri, J.cst, J.part,
                                                   J.stride, nullptr, 0, nullptr, nullptr);
        break;
      default:
        v2::me_slot<5, double, false, true, false>(nullptr, J.rec, e, slot, gc, J.tab, J.mask, J.ctri, J.cst, J.part,
                                                   J.stride, nullptr, 0, nullptr, nullptr);
        break;
    }
  }
}

}  // namespace pers
}  // namespace mg

namespace {

int64_t pad_pg(int64_t n) { return (n + mg::kPage - 1) / mg::kPage * mg::kPage; }

mg_status grow_d(double** buf, int64_t* cap, int64_t need) {
  if (need <= *cap) return MG_OK;
  if (*buf) mg::dev_free(*buf);
  *buf = nullptr;
  *cap = 0;
  if (mg::dev_alloc(buf, static_cast<size_t>(need) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return MG_ENOMEM;
  }
  *cap = need;
  return MG_OK;
}

}  // namespace

extern "C" mg_status mg_sigmakin_batch(const mg_batch_job* jobs, int njobs, void* stream) {
  if (!jobs || njobs < 1 || njobs > mg::pers::kMaxJobs) return MG_EINVAL;
  for (int i = 0; i < njobs; ++i) {
    const mg_batch_job& j = jobs[i];
    if (!j.ctx || j.nevt < 0 || (j.nevt > 0 && (!j.mom_dev || !j.me_dev))) return MG_EINVAL;
    if (j.ctx->prm.wt != 0.0) return MG_ENOTSUP;
    for (int k = 0; k < i; ++k)
      if (jobs[k].ctx == j.ctx) return MG_EINVAL;   // one context per job: the scratch is per context
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // per job: helicity mask (first call), scratch, per-event record; the tile table, costliest jobs first
  std::vector<int> order(njobs);
  for (int i = 0; i < njobs; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return jobs[a].ctx->K > jobs[b].ctx->K; });
  mg::pers::PBatch* batch = new (std::nothrow) mg::pers::PBatch;
  if (!batch) return MG_ENOMEM;
  batch->njobs = 0;
  batch->ntiles = 0;
  mg_status s = MG_OK;
  for (int oi = 0; oi < njobs && s == MG_OK; ++oi) {
    const mg_batch_job& j = jobs[order[oi]];
    mg_ctx* c = j.ctx;
    if (j.nevt == 0) continue;
    if (!c->mask_ready) s = mg_hel_filter(c, j.mom_dev, j.nevt, stream);
    const int64_t stride = pad_pg(j.nevt);
    if (s == MG_OK) s = grow_d(&c->d_part, &c->part_cap, stride * c->nhel);
    if (s == MG_OK) s = grow_d(&c->d_prep, &c->prep_cap, stride * mg::event_record_bytes(c->K, false) / 8 + 1);
    if (s != MG_OK) break;
    c->last = st;
    mg::MeConst cst;
    cst.gs = std::sqrt(4.0 * 3.14159265358979323846 * c->prm.alphas);
    cst.mt = c->prm.mt;
    cst.wt = c->prm.wt;
    cst.colour_scale = cst.gs * cst.gs / static_cast<double>(c->colour_den);
    if (mg::launch_event_prep(c->K, false, j.mom_dev, j.nevt, cst, c->d_prep, st) != cudaSuccess) { s = MG_ECUDA; break; }
    // the job's currents and quark-line prefixes shared between its gluon-helicity combinations, where its
    // context's FP64 shape asks for them and the whole job's buffer stays within 2 GiB
    const double* share = nullptr;
    const int64_t sdoubles = stride * mg::share_doubles(c->K);
    if (c->shape[MG_FP64].shared && sdoubles <= (int64_t(1) << 28)) {
      s = grow_d(&c->d_share, &c->share_cap, sdoubles);
      if (s != MG_OK) break;
      if (mg::launch_share(c->K, c->d_prep, j.nevt, c->d_tab, cst, c->d_share, st) != cudaSuccess) { s = MG_ECUDA; break; }
      share = c->d_share;
    }
    mg::pers::PJob& p = batch->job[batch->njobs++];
    p.share = share;
    p.rec = c->d_prep;
    p.tab = c->d_tab;
    p.gslots = c->d_gslots;
    p.nslot = c->d_ngslots;
    p.mask = c->d_mask;
    p.ctri = c->d_ctri;
    p.part = c->d_part;
    p.nevt = j.nevt;
    p.stride = stride;
    p.K = c->K;
    p.ntile_ev = static_cast<int>((j.nevt + mg::pers::kTileEv - 1) / mg::pers::kTileEv);
    p.tile0 = batch->ntiles;
    p.cst = cst;
    batch->ntiles += static_cast<int64_t>(p.ntile_ev) << c->K;   // every possible slot; absent ones exit at once
  }
  if (s == MG_OK && batch->njobs > 0) {
    // the tile counter of the costliest job's context (a context's work is ordered on one stream at a time)
    unsigned long long* counter_dev = jobs[order[0]].ctx->d_tiles;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mg::pers::k_me_persistent, mg::kMeThreads, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    int64_t blocks = static_cast<int64_t>(nsm) * per_sm;
    if (blocks > batch->ntiles) blocks = batch->ntiles;
    if (cudaMemsetAsync(counter_dev, 0, sizeof(unsigned long long), st) != cudaSuccess) s = MG_ECUDA;
    if (s == MG_OK) {
      mg::pers::k_me_persistent<<<static_cast<unsigned>(blocks), mg::kMeThreads, 0, st>>>(*batch, counter_dev);
      mg::note_launch();
      if (cudaGetLastError() != cudaSuccess) s = MG_ECUDA;
    }
    for (int i = 0; i < njobs && s == MG_OK; ++i) {
      const mg_batch_job& j = jobs[i];
      if (j.nevt == 0) continue;
      const double norm = 1.0 / (256.0 * mg::factorial(j.ctx->ng));
      if (mg::launch_hel_sum(j.ctx->d_part, j.ctx->d_ngslots, j.nevt, pad_pg(j.nevt), norm, j.me_dev, st) != cudaSuccess)
        s = MG_ECUDA;
    }
  }
  delete batch;
  return s;
}
