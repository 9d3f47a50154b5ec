// mg_tune.cu -- autotuner for the matrix-element launch shape, and CUDA-graph batches.
//
// Autotuner: for one context and precision, time mg_sigmakin on probe events for every launch
// shape of the matrix-element kernel (events per block 32 / 64 / 128, the remaining threads of the
// 128-thread block taking further gluon-helicity slots of the same events; grid dispatched event-
// tile-major or slot-tile-major) and keep the fastest.  Results can be cached in a text file, one
// line per (GPU, process, precision).
//
// Graph batches: the whole random numbers -> momenta -> matrix elements step (mg_rambo_range ->
// mg_hel_filter -> mg_sigmakin) of several jobs -- any mix of processes, one context each -- is
// captured once into a single CUDA graph, the jobs on parallel branches, and then replayed with
// one cudaGraphLaunch per batch.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mg_alloc.h"
#include "mg_ctx.h"
#include "mg_internal.h"
#include "mg_kernels.h"

namespace {

std::string cache_key(mg_ctx* ctx, mg_precision precision) {
  int dev = 0;
  cudaDeviceProp prop;
  std::memset(&prop, 0, sizeof(prop));
  if (cudaGetDevice(&dev) == cudaSuccess) cudaGetDeviceProperties(&prop, dev);
  std::string name(prop.name);
  for (char& c : name)
    if (c == ' ') c = '_';
  return name + "|" + std::to_string(static_cast<int>(ctx->proc)) + "|" + std::to_string(static_cast<int>(precision));
}

int launch_flags(const mg::MeShape& s) {
  return (s.unrolled ? MG_LAUNCH_UNROLLED : 0) | (s.df_redo ? MG_LAUNCH_DF_REDO : 0) | (s.fused ? MG_LAUNCH_FUSED : 0) |
         (s.warp ? MG_LAUNCH_WARP : 0) | (s.tc_apart ? MG_LAUNCH_TC_APART : 0) | (s.shared ? MG_LAUNCH_SHARED : 0) |
         (s.tc_sync ? MG_LAUNCH_TC_SYNC : 0);
}

bool cache_lookup(const char* path, const std::string& key, mg::MeShape* shape, double* ms) {
  if (!path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    char k[256];
    int tev = 0, sm = 0, un = 1;
    double t = 0;
    if (std::sscanf(line, "%255s %d %d %d %lf", k, &tev, &sm, &un, &t) != 5) continue;
    if (key == k && (tev == 32 || tev == 64 || tev == 128)) {
      shape->tile_ev = tev;
      shape->slot_major = sm != 0;
      shape->unrolled = (un & MG_LAUNCH_UNROLLED) != 0;
      shape->df_redo = (un & MG_LAUNCH_DF_REDO) != 0;
      shape->fused = (un & MG_LAUNCH_FUSED) != 0;
      shape->warp = (un & MG_LAUNCH_WARP) != 0;
      shape->tc_apart = (un & MG_LAUNCH_TC_APART) != 0;
      shape->shared = (un & MG_LAUNCH_SHARED) != 0;
      shape->tc_sync = (un & MG_LAUNCH_TC_SYNC) != 0;
      *ms = t;
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, const mg::MeShape& s, double ms) {
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %.6f\n", key.c_str(), s.tile_ev, s.slot_major ? 1 : 0, launch_flags(s), ms);
  std::fclose(f);
}

}  // namespace

extern "C" mg_status mg_autotune(mg_ctx* ctx, mg_precision precision, int64_t nevt, const char* cache_path,
                                 double* best_ms) {
  if (!ctx || nevt < 32 || precision < MG_FP64 || precision > MG_MIXED) return MG_EINVAL;
  const std::string key = cache_key(ctx, precision);
  mg::MeShape cached;
  double cms = 0;
  if (cache_lookup(cache_path, key, &cached, &cms)) {
    ctx->shape[precision] = cached;
    if (best_ms) *best_ms = cms;
    return MG_OK;
  }
  double* mom = nullptr;
  double* me = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mg_status rc = MG_OK;
  const mg::MeShape saved = ctx->shape[precision];
  if (mg::dev_alloc(&mom, mg_mom_count(ctx->proc, nevt) * sizeof(double)) != cudaSuccess ||
      mg::dev_alloc(&me, nevt * sizeof(double)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    rc = MG_ENOMEM;
  }
  mg::MeShape best = saved;
  float best_t = 1e30f;
  if (rc == MG_OK) rc = mg_rambo(ctx, 0x7E57, nevt, 1500.0, mom, nullptr, st);
  if (rc == MG_OK) rc = mg_hel_filter(ctx, mom, nevt, st);
  auto time_shape = [&](const mg::MeShape& s, float* out_ms) -> mg_status {
    ctx->shape[precision] = s;
    mg_status r = mg_sigmakin(ctx, mom, nevt, precision, me, st);   // warm-up (and scratch growth)
    float t = 1e30f;
    for (int rep = 0; rep < 3 && r == MG_OK; ++rep) {
      cudaEventRecord(e0, st);
      r = mg_sigmakin(ctx, mom, nevt, precision, me, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) { cudaGetLastError(); r = MG_ECUDA; break; }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < t) t = ms;
    }
    *out_ms = t;
    return r;
  };
  const int tiles[3] = {32, 64, 128};
  const bool fp32 = precision == MG_FP32_AMP || precision == MG_MIXED;
  const int nun = mg::me_static_available(ctx->K, fp32) && ctx->prm.wt == 0.0 ? 2 : 1;
  for (int un = 0; un < nun && rc == MG_OK; ++un)
    for (int ti = 0; ti < 3 && rc == MG_OK; ++ti)
      for (int sm = 0; sm < 2 && rc == MG_OK; ++sm) {
        mg::MeShape s;
        s.tile_ev = tiles[ti];
        s.slot_major = sm != 0;
        s.unrolled = nun == 2 ? un == 0 : true;
        s.fused = false;
        float t = 1e30f;
        rc = time_shape(s, &t);
        if (rc == MG_OK && t < best_t) { best_t = t; best = s; }
      }
  if (nun == 2 && rc == MG_OK) {   // the unrolled kernel with the record computed inside (fixed shape)
    mg::MeShape s;
    s.fused = true;
    float t = 1e30f;
    rc = time_shape(s, &t);
    if (rc == MG_OK && t < best_t) { best_t = t; best = s; }
  }
  if (mg::me_warp_available(ctx->K, fp32) && ctx->prm.wt == 0.0 && rc == MG_OK) {   // lane group per slot
    for (int apart = 0; apart < (precision == MG_MIXED ? 2 : 1) && rc == MG_OK; ++apart) {
      mg::MeShape s;
      s.warp = true;
      s.tc_apart = apart != 0;
      float t = 1e30f;
      rc = time_shape(s, &t);
      if (rc == MG_OK && t < best_t) { best_t = t; best = s; }
    }
  }
  if ((fp32 || precision == MG_FP64) && rc == MG_OK) {   // recomputation arithmetic / shared currents
    mg::MeShape s = best;
    if (fp32) s.df_redo = !s.df_redo;
    else s.shared = !s.shared;
    float t = 1e30f;
    rc = time_shape(s, &t);
    if (rc == MG_OK && t < best_t) { best_t = t; best = s; }
  }
  if ((precision == MG_FP64_TCCOLOR || precision == MG_MIXED) && rc == MG_OK) {   // colour-pass kernel
    mg::MeShape s = best;
    s.tc_sync = !s.tc_sync;
    float t = 1e30f;
    rc = time_shape(s, &t);
    if (rc == MG_OK && t < best_t) { best_t = t; best = s; }
  }
  ctx->shape[precision] = rc == MG_OK ? best : saved;
  if (rc == MG_OK) {
    cache_store(cache_path, key, best, best_t);
    if (best_ms) *best_ms = best_t;
  }
  if (st) cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (mom) mg::dev_free(mom);
  if (me) mg::dev_free(me);
  ctx->last = nullptr;
  return rc;
}

extern "C" mg_status mg_get_launch_shape(mg_ctx* ctx, mg_precision precision, int* tile_ev, int* slot_major,
                                         int* flags) {
  if (!ctx || precision < MG_FP64 || precision > MG_MIXED) return MG_EINVAL;
  if (tile_ev) *tile_ev = ctx->shape[precision].tile_ev;
  if (slot_major) *slot_major = ctx->shape[precision].slot_major ? 1 : 0;
  if (flags) *flags = launch_flags(ctx->shape[precision]);
  return MG_OK;
}

extern "C" mg_status mg_set_launch_shape(mg_ctx* ctx, mg_precision precision, int tile_ev, int slot_major,
                                         int flags) {
  if (!ctx || precision < MG_FP64 || precision > MG_MIXED) return MG_EINVAL;
  if ((tile_ev != 32 && tile_ev != 64 && tile_ev != 128) || (slot_major != 0 && slot_major != 1) ||
      (flags & ~(MG_LAUNCH_UNROLLED | MG_LAUNCH_DF_REDO | MG_LAUNCH_FUSED | MG_LAUNCH_WARP | MG_LAUNCH_TC_APART |
                 MG_LAUNCH_SHARED | MG_LAUNCH_TC_SYNC)) != 0)
    return MG_EINVAL;
  ctx->shape[precision].tile_ev = tile_ev;
  ctx->shape[precision].slot_major = slot_major != 0;
  ctx->shape[precision].unrolled = (flags & MG_LAUNCH_UNROLLED) != 0;
  ctx->shape[precision].df_redo = (flags & MG_LAUNCH_DF_REDO) != 0;
  ctx->shape[precision].fused = (flags & MG_LAUNCH_FUSED) != 0;
  ctx->shape[precision].warp = (flags & MG_LAUNCH_WARP) != 0;
  ctx->shape[precision].tc_apart = (flags & MG_LAUNCH_TC_APART) != 0;
  ctx->shape[precision].shared = (flags & MG_LAUNCH_SHARED) != 0;
  ctx->shape[precision].tc_sync = (flags & MG_LAUNCH_TC_SYNC) != 0;
  return MG_OK;
}

// ---------------------------------------------------------------------------------------------
// graph batches
// ---------------------------------------------------------------------------------------------
struct mg_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
  int flags = 0;
};

extern "C" void mg_graph_destroy(mg_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

namespace {

mg_status check_jobs(const mg_job* jobs, int njobs) {
  if (!jobs || njobs < 1 || njobs > 256) return MG_EINVAL;
  for (int i = 0; i < njobs; ++i) {
    const mg_job& j = jobs[i];
    if (!j.ctx || j.nevt < 1 || j.e0 < 0 || !j.mom_dev || !j.me_dev || j.precision < MG_FP64 || j.precision > MG_MIXED)
      return MG_EINVAL;
    for (int k = 0; k < i; ++k)
      if (jobs[k].ctx == j.ctx) return MG_EINVAL;   // one context per job: scratch is per context
    if ((j.precision == MG_FP64_TCCOLOR || j.precision == MG_MIXED) && j.ctx->prm.wt != 0.0) return MG_ENOTSUP;
  }
  // everything a captured call would allocate or configure happens now, outside the capture
  for (int i = 0; i < njobs; ++i) {
    mg_status s = mg::ctx_reserve(jobs[i].ctx, jobs[i].nevt, jobs[i].precision);
    if (s != MG_OK) return s;
    if (jobs[i].precision == MG_FP64_TCCOLOR || jobs[i].precision == MG_MIXED)
      if (mg::launch_colour_tc(jobs[i].ctx->ncol, nullptr, 0, jobs[i].ctx->nhel, nullptr, nullptr, 0.0, nullptr, 0,
                               nullptr) != cudaSuccess ||
          mg::launch_colour_umma(jobs[i].ctx->ncol, nullptr, 0, jobs[i].ctx->nhel, nullptr, nullptr, 0.0, nullptr, 0,
                                 nullptr, nullptr, nullptr) != cudaSuccess) {
        cudaGetLastError();
        return MG_ECUDA;
      }
  }
  return MG_OK;
}

// Capture the jobs into a new graph: a fork from one origin stream, each job's step on its own
// branch, a join back.
mg_status capture(const mg_job* jobs, int njobs, cudaGraph_t* out, bool persistent = false) {
  std::vector<cudaStream_t> streams(njobs, nullptr);
  std::vector<cudaEvent_t> done(njobs, nullptr);
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr;
  mg_status rc = MG_OK;
  if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess)
    rc = MG_ECUDA;
  for (int i = 0; i < njobs && rc == MG_OK; ++i)
    if (cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming) != cudaSuccess)
      rc = MG_ECUDA;
  bool capturing = false;
  if (rc == MG_OK && cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) == cudaSuccess) capturing = true;
  else if (rc == MG_OK) rc = MG_ECUDA;
  if (rc == MG_OK && cudaEventRecord(fork, origin) != cudaSuccess) rc = MG_ECUDA;
  for (int i = 0; i < njobs && rc == MG_OK; ++i) {
    const mg_job& j = jobs[i];
    if (cudaStreamWaitEvent(streams[i], fork, 0) != cudaSuccess) { rc = MG_ECUDA; break; }
    rc = mg_rambo_range(j.ctx, j.seed, j.e0, j.nevt, j.sqrts, j.mom_dev, nullptr, streams[i]);
    if (rc == MG_OK) rc = mg_hel_filter(j.ctx, j.mom_dev, j.nevt, streams[i]);
    if (rc == MG_OK && !persistent) rc = mg_sigmakin(j.ctx, j.mom_dev, j.nevt, j.precision, j.me_dev, streams[i]);
    if (rc == MG_OK && (cudaEventRecord(done[i], streams[i]) != cudaSuccess ||
                        cudaStreamWaitEvent(origin, done[i], 0) != cudaSuccess))
      rc = MG_ECUDA;
  }
  if (rc == MG_OK && persistent) {   // after every branch: all matrix elements in one persistent launch
    std::vector<mg_batch_job> b(njobs);
    for (int i = 0; i < njobs; ++i) b[i] = {jobs[i].ctx, jobs[i].mom_dev, jobs[i].nevt, jobs[i].me_dev};
    rc = mg_sigmakin_batch(b.data(), njobs, origin);
  }
  cudaGraph_t graph = nullptr;
  if (capturing && cudaStreamEndCapture(origin, &graph) != cudaSuccess && rc == MG_OK) rc = MG_ECUDA;
  cudaGetLastError();
  for (int i = 0; i < njobs; ++i) {
    jobs[i].ctx->last = nullptr;
    if (done[i]) cudaEventDestroy(done[i]);
    if (streams[i]) cudaStreamDestroy(streams[i]);
  }
  if (fork) cudaEventDestroy(fork);
  if (origin) cudaStreamDestroy(origin);
  if (rc != MG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  *out = graph;
  return MG_OK;
}

}  // namespace

extern "C" mg_status mg_graph_create(const mg_job* jobs, int njobs, mg_graph** out) {
  return mg_graph_create_ex(jobs, njobs, 0, out);
}

extern "C" mg_status mg_graph_create_ex(const mg_job* jobs, int njobs, int flags, mg_graph** out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  if (flags & ~MG_GRAPH_PERSISTENT) return MG_EINVAL;
  const bool persistent = (flags & MG_GRAPH_PERSISTENT) != 0;
  mg_status rc = check_jobs(jobs, njobs);
  if (rc != MG_OK) return rc;
  if (persistent) {
    if (njobs > 64) return MG_EINVAL;
    for (int i = 0; i < njobs; ++i)
      if (jobs[i].precision != MG_FP64 || jobs[i].ctx->prm.wt != 0.0) return MG_ENOTSUP;
  }
  mg_graph* g = new (std::nothrow) mg_graph;
  if (!g) return MG_ENOMEM;
  g->flags = flags;
  rc = capture(jobs, njobs, &g->graph, persistent);
  if (rc == MG_OK && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) { cudaGetLastError(); rc = MG_ECUDA; }
  if (rc == MG_OK) {
    size_t n = 0;
    if (cudaGraphGetNodes(g->graph, nullptr, &n) == cudaSuccess) g->launches = static_cast<int>(n);
  }
  if (rc != MG_OK) {
    mg_graph_destroy(g);
    return rc;
  }
  *out = g;
  return MG_OK;
}

extern "C" mg_status mg_graph_update(mg_graph* g, const mg_job* jobs, int njobs) {
  if (!g || !g->exec) return MG_EINVAL;
  mg_status rc = check_jobs(jobs, njobs);
  if (rc != MG_OK) return rc;
  if (g->flags & MG_GRAPH_PERSISTENT)
    for (int i = 0; i < njobs; ++i)
      if (jobs[i].precision != MG_FP64 || jobs[i].ctx->prm.wt != 0.0) return MG_ENOTSUP;
  cudaGraph_t ng = nullptr;
  rc = capture(jobs, njobs, &ng, (g->flags & MG_GRAPH_PERSISTENT) != 0);
  if (rc != MG_OK) return rc;
  cudaGraphExecUpdateResultInfo info;
  if (cudaGraphExecUpdate(g->exec, ng, &info) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(ng);
    return MG_EINVAL;   // topology changed (different jobs): create a new graph
  }
  cudaGraphDestroy(g->graph);
  g->graph = ng;
  return MG_OK;
}

extern "C" mg_status mg_graph_launch(mg_graph* g, void* stream) {
  if (!g || !g->exec) return MG_EINVAL;
  if (cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    cudaGetLastError();
    return MG_ECUDA;
  }
  return MG_OK;
}

extern "C" mg_status mg_graph_nodes(mg_graph* g, int* nodes) {
  if (!g || !nodes) return MG_EINVAL;
  *nodes = g->launches;
  return MG_OK;
}
