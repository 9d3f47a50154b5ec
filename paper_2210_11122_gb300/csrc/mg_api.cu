// mg_api.cu -- the C ABI of include/mg.h: contexts, argument checks, launches, error handling.
//
// Host runtime for the paper's workflow (Sec. 1, Fig. 1): random numbers -> momenta -> matrix
// elements, every step a kernel on the current CUDA device, stream-ordered and asynchronous.
// No C++ exception crosses the ABI; every entry point returns an mg_status.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "mg_alloc.h"
#include "mg_ctx.h"
#include "mg_internal.h"
#include "mg_kernels.h"

namespace {

const double kPi = 3.14159265358979323846;

#define MG_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return MG_ECUDA;             \
  } while (0)

bool valid_proc(mg_process p) { return p >= MG_GG_TT && p <= MG_GG_TTGGG; }

int64_t pad32(int64_t n) { return (n + mg::kPage - 1) / mg::kPage * mg::kPage; }

mg_status grow(double** buf, int64_t* cap, int64_t need) {
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

// Flop model of the matrix-element kernel of mg_me2.cu for one event (FMA counted as 2 flops, a
// complex multiply-add as 8): mirrors the kernel operation by operation.  One thread per gluon-
// helicity combination with a good helicity; per thread the gluon currents once, (gamma.J) v per
// antitop helicity, a depth-first walk of the quark-line prefixes per top helicity, the jamps and
// the colour sum per good helicity.  mask == NULL means every helicity is good.
// warp_simt: the FP32 lane-group kernel's SIMT colour epilogue, which multiplies the full ncol x ncol matrix
// into the jamps of all four helicities of a slot (4 ncol^2 + 4 ncol each, good or not) instead of the
// packed triangle per good helicity.  warp: the FP32 lane-group kernel (any epilogue), which for 5 gluons
// takes the gluon-pair currents from the record; the FP32 record of 5 gluons computes them in FP64.
void flop_model(const mg::Tables& t, const uint32_t* mask, bool fp32, bool shared, bool warp, bool warp_simt,
                double* amp, double* col) {
  const int K = t.K, nsub = 1 << K, npar = K + 2;
  // three-gluon vertex in the current-conserving form: d (4) + JL.JR (30) + JL.PR, JR.PL (2 x 14) +
  // two scalings (4) + 4 x (real-complex and two complex multiply-adds) (80)
  const double v3 = 146.0, v4 = 192.0, row_gamma = 72.0, row_prop = 56.0, gamma_col = 64.0, sdot = 32.0,
               mdot = 30.0;
  const bool pairs = fp32 && K == 5;                              // gluon-pair currents in the FP32 record
  const double per_event = 25.0 * nsub + 30.0 * K + 100.0 +      // subsets, propagators, wavefunctions (once)
                           (pairs ? K * (K - 1) / 2 * (4.0 * (v3 + 8.0) + 20.0) : 0.0);
  double per_slot = 0.0;                                           // gluon currents of one helicity combination
  double shared_work = 0.0;                                        // (shared: once per event)
  for (int s = K; s < t.nseq; ++s) {
    const double c = v3 * t.seq_nv3[s] + v4 * t.seq_nv4[s] + 8.0;
    if (shared) shared_work += c * (1 << t.seq_len[s]);   // once per helicity assignment of its own gluons
    else if (!(pairs && warp && t.seq_len[s] == 2)) per_slot += c;
  }
  for (int f = 0; f < t.nfull; ++f) per_slot += v3 * t.full_nv3[f] + v4 * t.full_nv4[f] + 8.0;
  // FP64: (gamma.J) v tabulated for every current and both antitop helicities; FP32: formed per jamp term
  if (!fp32) {
    if (shared)
      for (int s = 0; s < t.nseq; ++s) shared_work += 2.0 * gamma_col * (1 << t.seq_len[s]);
    else
      per_slot += 2.0 * gamma_col * t.nseq;
  }
  // shared (FP64): the quark-line prefixes of lengths 1 .. pref_levels once per helicity assignment of
  // their gluons and top helicity per event (k_prefix_level: both top helicities share each current's
  // gamma.J entries, the 8 additions of row_gamma), the longer ones in the slot's walk
  const int plev = shared ? t.pref_levels : 0;
  for (int m = 1; m <= plev; ++m) {
    int orderings = 1;
    for (int i = 0; i < m; ++i) orderings *= K - i;
    shared_work += static_cast<double>(orderings << m) * (8.0 * m + 2.0 * ((row_gamma - 8.0) * m + row_prop));
  }
  double walk = 50.0 + 2.0 * 72.0;                                 // ubar, two quark currents
  for (int c = 0; c < t.ncol; ++c) {
    for (int m = t.lcp[c] + 1; m < K; ++m) walk += m <= plev ? 0.0 : row_gamma * m + row_prop;
    walk += fp32 ? 2.0 * mdot + (K - 1) * (row_gamma + 2.0 * sdot)  // jamps of both antitop helicities
                 : 2.0 * (mdot + sdot * (K - 1));
  }
  const double colour = 4.0 * t.ncol * (t.ncol + 1) / 2.0 + 4.0 * t.ncol;
  double a = per_event + shared_work, c = 0;
  for (int gc = 0; gc < nsub; ++gc) {
    int hb = 0;
    for (int g = 0; g < K; ++g)
      if ((gc >> g) & 1) hb |= 1 << (npar - 1 - (g < 2 ? g : g + 2));
    int good[4], any = 0;
    for (int k = 0; k < 4; ++k) {
      const int h = hb | ((k >> 1) << (npar - 3)) | ((k & 1) << (npar - 4));   // k = 2*top + antitop
      good[k] = mask ? static_cast<int>((mask[h >> 5] >> (h & 31)) & 1u) : 1;
      any |= good[k];
    }
    if (!any) continue;
    a += per_slot;
    for (int top = 0; top < 2; ++top)
      if (good[2 * top] || good[2 * top + 1]) a += walk;
    if (warp_simt)
      c += 4.0 * (4.0 * t.ncol * t.ncol + 4.0 * t.ncol);
    else
      for (int k = 0; k < 4; ++k) c += good[k] ? colour : 0.0;
  }
  *amp = a;
  *col = c;
}

mg_status grow_repair(mg_ctx* ctx, int64_t n) {
  if (!ctx->d_nrepair) {
    if (mg::dev_alloc(&ctx->d_nrepair, sizeof(int)) != cudaSuccess) { cudaGetLastError(); return MG_ENOMEM; }
  }
  if (n <= ctx->repair_cap) return MG_OK;
  if (ctx->d_repair) mg::dev_free(ctx->d_repair);
  if (ctx->d_flag) mg::dev_free(ctx->d_flag);
  ctx->d_repair = nullptr;
  ctx->d_flag = nullptr;
  ctx->repair_cap = 0;
  if (mg::dev_alloc(&ctx->d_repair, static_cast<size_t>(n) * sizeof(int)) != cudaSuccess ||
      mg::dev_alloc(&ctx->d_flag, static_cast<size_t>(n)) != cudaSuccess) {
    cudaGetLastError();
    return MG_ENOMEM;
  }
  ctx->repair_cap = n;
  return MG_OK;
}

}  // namespace

namespace mg {

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// allocations: live count, and the countdown of the injected failure (0: none armed)
static std::atomic<int64_t> g_live_allocs{0};
static std::atomic<int64_t> g_fail_countdown{0};

cudaError_t alloc_raw(void** p, size_t bytes, bool host) {
  int64_t n = g_fail_countdown.load();
  while (n > 0 && !g_fail_countdown.compare_exchange_weak(n, n - 1)) {
  }
  if (n == 1) {   // this call brought the countdown to zero: it fails, as an exhausted device would
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  const cudaError_t e = host ? cudaMallocHost(p, bytes) : cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_live_allocs.fetch_add(1);
  return e;
}

cudaError_t free_raw(void* p, bool host) {
  if (!p) return cudaSuccess;
  g_live_allocs.fetch_sub(1);
  return host ? cudaFreeHost(p) : cudaFree(p);
}

int64_t share_chunk(int K, int64_t stride) {
  const int64_t per_event = share_doubles(K);   // doubles
  int64_t chunk = (int64_t(1) << 28) / per_event / kPage * kPage;       // 2^28 doubles = 2 GiB
  if (chunk < kPage) chunk = kPage;
  return chunk < stride ? chunk : stride;
}

bool mixed_in_kernel(const mg_ctx* ctx, mg_precision precision) {
  return precision == MG_MIXED && ctx->prm.wt == 0.0 && ctx->shape[precision].warp &&
         !ctx->shape[precision].tc_apart && me_warp_available(ctx->K, true);
}

// Grow every scratch buffer of ctx so that mg_hel_filter and mg_sigmakin(precision) on up to nevt
// events allocate nothing (used by the serving loop, which must not synchronise the device).
mg_status ctx_reserve(mg_ctx* ctx, int64_t nevt, mg_precision precision) {
  if (!ctx || nevt < 1) return MG_EINVAL;
  const int64_t stride = pad32(nevt);
  const int64_t wstride = pad32(nevt < ctx->prm.hel_warmup ? nevt : ctx->prm.hel_warmup);
  mg_status s = grow(&ctx->d_part, &ctx->part_cap, (stride > wstride ? stride : wstride) * ctx->nhel);
  if (s == MG_OK) s = grow(&ctx->d_tot, &ctx->tot_cap, wstride);
  const bool fp32 = precision == MG_FP32_AMP || precision == MG_MIXED;
  const bool tc = (precision == MG_FP64_TCCOLOR || precision == MG_MIXED) && !mixed_in_kernel(ctx, precision);
  int64_t chunk = stride;
  if (tc) {
    const int64_t per_event = static_cast<int64_t>(ctx->nhel) * ctx->ncol;
    chunk = (int64_t(1) << 29) / per_event / kPage * kPage;
    if (chunk < kPage) chunk = kPage;
    if (chunk > stride) chunk = stride;
    if (s == MG_OK && ctx->jamp_cap < chunk * per_event) {
      if (ctx->d_jamps) mg::dev_free(ctx->d_jamps);
      ctx->d_jamps = nullptr;
      ctx->jamp_cap = 0;
      if (mg::dev_alloc(&ctx->d_jamps, static_cast<size_t>(chunk * per_event) * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        return MG_ENOMEM;
      }
      ctx->jamp_cap = chunk * per_event;
    }
  }
  if (s == MG_OK) s = grow(&ctx->d_prep, &ctx->prep_cap, chunk * event_record_bytes(ctx->K, fp32) / 8 + 1);
  if (s == MG_OK) s = grow_repair(ctx, chunk);
  if (s == MG_OK && (precision == MG_FP64 || precision == MG_FP64_TCCOLOR) && ctx->shape[precision].shared &&
      ctx->prm.wt == 0.0) {
    const int64_t sc = share_chunk(ctx->K, stride);
    s = grow(&ctx->d_share, &ctx->share_cap, (sc < chunk ? sc : chunk) * share_doubles(ctx->K));
  }
  return s;
}

mg_status ctx_copy_mask(mg_ctx* dst, const mg_ctx* src, cudaStream_t st) {
  if (!dst || !src || dst->proc != src->proc) return MG_EINVAL;
  auto cp = [&](void* d, const void* s, size_t n) {
    return cudaMemcpyAsync(d, s, n, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
  };
  const bool ok = cp(dst->d_mask, src->d_mask, 4 * sizeof(uint32_t)) && cp(dst->d_good, src->d_good, 128 * sizeof(int)) &&
                  cp(dst->d_ngood, src->d_ngood, sizeof(int)) && cp(dst->d_maxr, src->d_maxr, 128 * sizeof(double)) &&
                  cp(dst->d_gslots, src->d_gslots, 32 * sizeof(int)) && cp(dst->d_ngslots, src->d_ngslots, sizeof(int)) &&
                  cp(dst->d_nrows, src->d_nrows, sizeof(int));
  if (!ok) { cudaGetLastError(); return MG_ECUDA; }
  dst->mask_ready = true;
  return MG_OK;
}

// Device bytes one sigmakin call of nevt events touches (momenta, MEs, scratch): the serving
// loop's admission footprint.
int64_t footprint_bytes(mg_process proc, int64_t nevt, mg_precision precision) {
  const int K = gluons_of(proc), npar = K + 2, nhel = 1 << npar, ncol = factorial(K);
  const int64_t stride = pad32(nevt);
  const bool fp32 = precision == MG_FP32_AMP || precision == MG_MIXED;
  // jamps in device memory: the tensor-core colour modes, except FP32 amplitudes with four or five
  // gluons, whose default lane-group kernel sums the colours on the tensor cores itself
  const bool tc = precision == MG_FP64_TCCOLOR || (precision == MG_MIXED && !me_warp_available(K, true)) ||
                  (precision == MG_MIXED && K < 4);
  int64_t b = stride * npar * 4 * 8 + stride * 8 + stride * nhel * 8 + stride * event_record_bytes(K, fp32);
  if (fp32) b += stride * (sizeof(int) + 1);   // recomputation list and flags
  if (tc) b += stride * nhel * ncol * 8;
  return b;
}

}  // namespace mg

extern "C" {

const char* mg_strerror(mg_status s) {
  switch (s) {
    case MG_OK: return "ok";
    case MG_EINVAL: return "invalid argument";
    case MG_ENOMEM: return "out of memory";
    case MG_ECUDA: return "CUDA error";
    case MG_ENOCONV: return "RAMBO did not converge";
    case MG_EAGAIN: return "not ready";
    case MG_ETIMEOUT: return "timed out";
    case MG_EBUSY: return "busy";
    case MG_ENOTSUP: return "not supported";
    case MG_ECANCELED: return "cancelled";
  }
  return "unknown status";
}

void mg_default_params(mg_params* p) {
  if (!p) return;
  p->mt = 173.0;
  p->wt = 0.0;
  p->alphas = 0.118;
  p->hel_warmup = 1024;
  p->hel_tau = 1e-9;
}

mg_status mg_process_info(mg_process proc, int* npar, int* nhel, int* ncol, int* ndiagrams) {
  if (!valid_proc(proc)) return MG_EINVAL;
  static const int nd[4] = {3, 16, 123, 1240};
  int K = mg::gluons_of(proc);
  if (npar) *npar = K + 2;
  if (nhel) *nhel = 1 << (K + 2);
  if (ncol) *ncol = mg::factorial(K);
  if (ndiagrams) *ndiagrams = nd[proc];
  return MG_OK;
}

int64_t mg_mom_count(mg_process proc, int64_t nevt) {
  if (!valid_proc(proc) || nevt < 0) return -1;
  return pad32(nevt) * mg::npar_of(proc) * 4;
}

mg_status mg_colour_matrix(mg_process proc, int64_t* num, int64_t* den) {
  if (!valid_proc(proc) || !num || !den) return MG_EINVAL;
  std::vector<int64_t> v;
  int64_t d;
  try {
    mg::colour_matrix_exact(mg::gluons_of(proc), v, d);
  } catch (...) {
    return MG_ENOMEM;
  }
  std::memcpy(num, v.data(), v.size() * sizeof(int64_t));
  *den = d;
  return MG_OK;
}

mg_status mg_flops_per_event_shape(mg_process proc, mg_precision precision, const uint32_t* mask, int flags,
                                   double* amp_flops, double* colour_flops) {
  if (!valid_proc(proc) || precision < MG_FP64 || precision > MG_MIXED) return MG_EINVAL;
  mg::Tables* t = new (std::nothrow) mg::Tables;
  if (!t) return MG_ENOMEM;
  mg::build_tables(mg::gluons_of(proc), *t);
  double a, c;
  const bool fp32 = precision == MG_FP32_AMP || precision == MG_MIXED;
  // flags < 0: the default algorithm of each mode (as mg_create's launch shapes): FP64 amplitudes share
  // the currents of fewer than all gluons between gluon-helicity combinations from 1 final-state gluon on
  const int K = mg::gluons_of(proc);
  const bool shared = flags < 0 ? K >= 3 : (flags & MG_LAUNCH_SHARED) != 0;
  // the lane-group kernel (FP32 amplitudes, 3..5 gluons; the default for 4 and 5) with its SIMT colour
  // epilogue: MG_FP32_AMP, or MG_MIXED whose colour sums then run on the tensor cores (not counted here)
  const bool warp = flags < 0 ? K >= 4 : (flags & MG_LAUNCH_WARP) != 0;
  const bool warp_fp32 = fp32 && warp && mg::me_warp_available(K, true);
  const bool warp_simt = precision == MG_FP32_AMP && warp_fp32;
  flop_model(*t, mask, fp32, !fp32 && shared, warp_fp32, warp_simt, &a, &c);
  delete t;
  if (amp_flops) *amp_flops = a;
  if (colour_flops) *colour_flops = c;
  return MG_OK;
}

mg_status mg_flops_per_event(mg_process proc, mg_precision precision, const uint32_t* mask, double* amp_flops,
                             double* colour_flops) {
  return mg_flops_per_event_shape(proc, precision, mask, -1, amp_flops, colour_flops);
}

void mg_destroy(mg_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  mg::dev_free(ctx->d_tab);
  mg::dev_free(ctx->d_ctri);
  mg::dev_free(ctx->d_ctri_f);
  mg::dev_free(ctx->d_cfull);
  mg::dev_free(ctx->d_mask);
  mg::dev_free(ctx->d_maxr);
  mg::dev_free(ctx->d_good);
  mg::dev_free(ctx->d_ngood);
  mg::dev_free(ctx->d_allhel);
  mg::dev_free(ctx->d_nhel);
  mg::dev_free(ctx->d_gslots);
  mg::dev_free(ctx->d_ngslots);
  mg::dev_free(ctx->d_allg);
  mg::dev_free(ctx->d_nrows);
  mg::dev_free(ctx->d_cmat);
  mg::dev_free(ctx->d_cumma);
  mg::dev_free(ctx->d_tcerr);
  mg::dev_free(ctx->d_tiles);
  mg::dev_free(ctx->d_jamps);
  mg::dev_free(ctx->d_nallg);
  mg::dev_free(ctx->d_nbad);
  mg::dev_free(ctx->d_part);
  mg::dev_free(ctx->d_tot);
  mg::dev_free(ctx->d_prep);
  mg::dev_free(ctx->d_repair);
  mg::dev_free(ctx->d_nrepair);
  mg::dev_free(ctx->d_flag);
  mg::dev_free(ctx->d_share);
  mg::dev_free(ctx->d_j2);
  mg::dev_free(ctx->d_sdetab);
  mg::dev_free(ctx->d_sde);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  mg::dev_free(ctx->d_mom_stage);
  mg::dev_free(ctx->d_me_stage);
  for (int c = 0; c < mg_ctx::kHostChunks; ++c) {
    if (ctx->ev_in[c]) cudaEventDestroy(ctx->ev_in[c]);
    if (ctx->ev_done[c]) cudaEventDestroy(ctx->ev_done[c]);
  }
  if (ctx->cp_in) cudaStreamDestroy(ctx->cp_in);
  if (ctx->cp_out) cudaStreamDestroy(ctx->cp_out);
  delete ctx;
}

mg_status mg_create(mg_process proc, const mg_params* params, mg_ctx** out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  if (!valid_proc(proc)) return MG_EINVAL;
  mg_params prm;
  mg_default_params(&prm);
  if (params) prm = *params;
  if (!(prm.mt >= 0.0) || !(prm.wt >= 0.0) || !(prm.alphas > 0.0) || prm.hel_warmup < 1 || !(prm.hel_tau >= 0.0))
    return MG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return MG_ECUDA; }
  mg_ctx* c = new (std::nothrow) mg_ctx;
  if (!c) return MG_ENOMEM;
  c->proc = proc;
  c->K = mg::gluons_of(proc);
  c->ng = c->K - 2;
  c->npar = c->K + 2;
  c->nhel = 1 << c->npar;
  c->ncol = mg::factorial(c->K);
  c->prm = prm;
  mg_status st = MG_OK;
  do {
    mg::Tables* t = new (std::nothrow) mg::Tables;
    if (!t) { st = MG_ENOMEM; break; }
    mg::build_tables(c->K, *t);
    cudaError_t e = mg::dev_alloc(&c->d_tab, sizeof(mg::Tables));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_tab, t, sizeof(mg::Tables), cudaMemcpyHostToDevice);
    delete t;
    if (e != cudaSuccess) { st = e == cudaErrorMemoryAllocation ? MG_ENOMEM : MG_ECUDA; break; }
    std::vector<int64_t> num;
    mg::colour_matrix_exact(c->K, num, c->colour_den);
    std::vector<double> tri;
    for (int a = 0; a < c->ncol; ++a)
      for (int b = a; b < c->ncol; ++b)
        tri.push_back(static_cast<double>(num[static_cast<size_t>(a) * c->ncol + b]) * (a == b ? 1.0 : 2.0));
    e = mg::dev_alloc(&c->d_ctri, tri.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_ctri, tri.data(), tri.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mg::me_static_upload_colour(c->K, tri.data(), static_cast<int>(tri.size()));
    std::vector<float> full(num.begin(), num.end());
    if (e == cudaSuccess) e = mg::dev_alloc(&c->d_cfull, full.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_cfull, full.data(), full.size() * sizeof(float), cudaMemcpyHostToDevice);
    std::vector<float> trif(tri.begin(), tri.end());
    if (e == cudaSuccess) e = mg::dev_alloc(&c->d_ctri_f, trif.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_ctri_f, trif.data(), trif.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { st = e == cudaErrorMemoryAllocation ? MG_ENOMEM : MG_ECUDA; break; }
    std::vector<int> all(c->nhel);
    for (int h = 0; h < c->nhel; ++h) all[h] = h;
    if (mg::dev_alloc(&c->d_mask, 4 * sizeof(uint32_t)) != cudaSuccess || mg::dev_alloc(&c->d_good, 128 * sizeof(int)) != cudaSuccess ||
        mg::dev_alloc(&c->d_maxr, 128 * sizeof(double)) != cudaSuccess ||
        mg::dev_alloc(&c->d_ngood, sizeof(int)) != cudaSuccess || mg::dev_alloc(&c->d_allhel, c->nhel * sizeof(int)) != cudaSuccess ||
        mg::dev_alloc(&c->d_nhel, sizeof(int)) != cudaSuccess || mg::dev_alloc(&c->d_nbad, sizeof(unsigned long long)) != cudaSuccess) {
      st = MG_ENOMEM;
      break;
    }
    const int ng2 = 1 << c->K;
    {
      std::vector<uint16_t> halves(mg::colour_tc_cmat_halves(c->ncol));
      mg::colour_tc_pack(c->ncol, num.data(), halves.data());
      std::vector<uint16_t> uh(mg::colour_umma_halves(c->ncol));
      mg::colour_umma_pack(c->ncol, num.data(), uh.data());
      if (mg::dev_alloc(&c->d_cumma, uh.size() * sizeof(uint16_t)) != cudaSuccess ||
          cudaMemcpy(c->d_cumma, uh.data(), uh.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess ||
          mg::dev_alloc(&c->d_tcerr, sizeof(int)) != cudaSuccess || cudaMemset(c->d_tcerr, 0, sizeof(int)) != cudaSuccess ||
          mg::dev_alloc(&c->d_tiles, sizeof(unsigned long long)) != cudaSuccess) {
        st = MG_ENOMEM;
        break;
      }
      if (mg::dev_alloc(&c->d_cmat, halves.size() * sizeof(uint16_t)) != cudaSuccess ||
          cudaMemcpy(c->d_cmat, halves.data(), halves.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess ||
          mg::dev_alloc(&c->d_nrows, sizeof(int)) != cudaSuccess || cudaMemset(c->d_nrows, 0, sizeof(int)) != cudaSuccess) {
        st = MG_ENOMEM;
        break;
      }
    }
    if (mg::dev_alloc(&c->d_gslots, 32 * sizeof(int)) != cudaSuccess || mg::dev_alloc(&c->d_ngslots, sizeof(int)) != cudaSuccess ||
        mg::dev_alloc(&c->d_allg, 32 * sizeof(int)) != cudaSuccess || mg::dev_alloc(&c->d_nallg, sizeof(int)) != cudaSuccess) {
      st = MG_ENOMEM;
      break;
    }
    if (cudaMemcpy(c->d_allg, all.data(), ng2 * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_nallg, &ng2, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->d_ngslots, 0, sizeof(int)) != cudaSuccess) {
      st = MG_ECUDA;
      break;
    }
    if (cudaMemcpy(c->d_allhel, all.data(), c->nhel * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_nhel, &c->nhel, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->d_nbad, 0, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(c->d_mask, 0, 4 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(c->d_ngood, 0, sizeof(int)) != cudaSuccess) {
      st = MG_ECUDA;
      break;
    }
    // four and five gluons: the FP32 modes default to the lane-group-per-slot kernel (the per-thread
    // state does not fit on chip); the autotuner can change it
    if (c->K >= 4)
      for (int p = 0; p < 4; ++p) c->shape[p].warp = true;
    // five gluons, FP32 amplitudes + tensor-core colour: the separate colour pass (measured 2 % faster
    // than the in-kernel one there); the autotuner can change it
    if (c->K == 5) c->shape[MG_MIXED].tc_apart = true;
    // FP64 amplitudes: share the currents of fewer than all gluons between gluon-helicity combinations
    // where that was measured faster (1, 2 and 3 final-state gluons); the autotuner can change it
    for (int p = 0; p < 4; ++p) c->shape[p].shared = c->K >= 3;
    // FP32 recomputation threshold: the largest plain-FP32 error among the events kept in FP32 was
    // measured at 3.6e-6 / 3.7e-6 (1 / 2 final-state gluons) with tau = 3e-4, and for 3 gluons, whose
    // lane-group kernel takes the gluon-pair currents from the FP64 record, at 3.9e-6 with tau = 3e-5,
    // which recomputes a twelfth as many events as 3e-4
    c->fp32_tau = c->K == 5 ? 3e-5 : 3e-4;
    // side stream of the FP32 modes' recomputation: highest priority, so that its few blocks are
    // dispatched ahead of the FP32 launch's
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      st = MG_ECUDA;
      break;
    }
  } while (false);
  if (st != MG_OK) {
    cudaGetLastError();
    mg_destroy(c);
    return st;
  }
  *out = c;
  return MG_OK;
}

mg_status mg_philox(uint64_t seed, int64_t nevt, int nfinal, uint32_t* words_dev, void* stream) {
  if (nevt < 0 || nfinal < 1 || nfinal > 64 || (nevt > 0 && !words_dev)) return MG_EINVAL;
  if (reinterpret_cast<uintptr_t>(words_dev) & 15u) return MG_EINVAL;
  if (nevt == 0) return MG_OK;
  MG_CUDA(mg::launch_philox(seed, nevt, nfinal, words_dev, static_cast<cudaStream_t>(stream)));
  return MG_OK;
}

mg_status mg_rambo(mg_ctx* ctx, uint64_t seed, int64_t nevt, double sqrts, double* mom_dev, double* wgt_dev,
                   void* stream) {
  return mg_rambo_range(ctx, seed, 0, nevt, sqrts, mom_dev, wgt_dev, stream);
}

mg_status mg_rambo_range(mg_ctx* ctx, uint64_t seed, int64_t e0, int64_t nevt, double sqrts, double* mom_dev,
                         double* wgt_dev, void* stream) {
  if (!ctx || nevt < 0 || e0 < 0 || (nevt > 0 && !mom_dev)) return MG_EINVAL;
  if (!(sqrts > 2.0 * ctx->prm.mt) || !std::isfinite(sqrts)) return MG_EINVAL;
  if (nevt == 0) return MG_OK;
  const int n = ctx->K;   // final-state particles
  double w0 = std::pow(2.0 * kPi, 4 - 3 * n) * std::pow(kPi / 2.0, n - 1) * std::pow(sqrts * sqrts, n - 2) /
              (mg::factorial(n - 1) * static_cast<double>(mg::factorial(n - 2)));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ctx->last = st;
  MG_CUDA(mg::launch_rambo(ctx->K, seed, e0, nevt, sqrts, ctx->prm.mt, w0, mom_dev, wgt_dev, ctx->d_nbad, st));
  return MG_OK;
}

static mg::MeConst me_const(const mg_ctx* ctx) {
  mg::MeConst c;
  c.gs = std::sqrt(4.0 * kPi * ctx->prm.alphas);
  c.mt = ctx->prm.mt;
  c.wt = ctx->prm.wt;
  c.colour_scale = c.gs * c.gs / static_cast<double>(ctx->colour_den);
  c.fp32_tau = ctx->fp32_tau;
  return c;
}

mg_status mg_set_fp32_tau(mg_ctx* ctx, double tau) {
  if (!ctx || !(tau >= 0.0) || !std::isfinite(tau)) return MG_EINVAL;
  ctx->fp32_tau = tau;
  return MG_OK;
}

mg_status mg_hel_filter(mg_ctx* ctx, const double* mom_dev, int64_t nevt, void* stream) {
  if (!ctx || nevt < 1 || !mom_dev) return MG_EINVAL;
  const int64_t w = nevt < ctx->prm.hel_warmup ? nevt : ctx->prm.hel_warmup;
  const int64_t stride = pad32(w);
  mg_status s = grow(&ctx->d_part, &ctx->part_cap, stride * ctx->nhel);
  if (s != MG_OK) return s;
  s = grow(&ctx->d_tot, &ctx->tot_cap, stride);
  if (s != MG_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ctx->last = st;
  const mg::MeConst cst = me_const(ctx);
  if (ctx->prm.wt == 0.0) {
    // FP32 amplitudes: the accepted and rejected helicities' ratios are at least six decades apart (the
    // kept ones >= 1e-6, the vanishing ones <= 1e-25 in FP64), far more than FP32 rounding can move a
    // ratio, so the mask is the one FP64 gives, at the FP32 pipe's rate
    MG_CUDA(mg::launch_me_gluonhel(ctx->K, true, true, mom_dev, nullptr, w, ctx->d_tab, ctx->d_allg, 1 << ctx->K,
                                   ctx->d_nallg, ctx->d_mask, ctx->d_ctri, ctx->d_ctri_f, cst, ctx->d_part, stride, st));
  } else {
    MG_CUDA(mg::launch_me_helicity(ctx->K, false, mom_dev, w, ctx->d_tab, ctx->d_allhel, ctx->nhel, ctx->d_nhel,
                                   ctx->d_ctri, cst, ctx->d_part, stride, st));
  }
  MG_CUDA(mg::launch_hel_sum(ctx->d_part, ctx->d_nhel, w, stride, 1.0, ctx->d_tot, st));
  MG_CUDA(mg::launch_hel_mask(ctx->d_part, ctx->d_tot, ctx->nhel, w, stride, ctx->prm.hel_tau, ctx->d_maxr,
                              ctx->d_mask, ctx->d_good, ctx->d_ngood, st));
  MG_CUDA(mg::launch_gluon_slots(ctx->d_mask, ctx->K, ctx->d_gslots, ctx->d_ngslots, ctx->d_nrows, st));
  ctx->mask_ready = true;
  return MG_OK;
}

// The FP32 modes' recomputation (double-float or FP64 amplitudes) of the events listed in
// ctx->d_repair, forked onto ctx->side after the work already queued on st (the per-event records and
// the list), and joined back.
static cudaError_t fork_repair(mg_ctx* ctx, const double* mom, int64_t nevt, const mg::MeConst& cst, int64_t stride,
                               int rows_out, bool df, cudaStream_t st) {
  cudaError_t e = cudaEventRecord(ctx->ev_fork, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
  if (e == cudaSuccess && df)
    e = mg::launch_me_repair(ctx->K, mom, nevt, ctx->d_tab, ctx->d_gslots, 1 << ctx->K, ctx->d_ngslots, ctx->d_mask,
                             ctx->d_ctri_f, ctx->d_cfull, cst, ctx->d_part, stride, ctx->d_repair, ctx->d_nrepair, rows_out,
                             ctx->side);
  else if (e == cudaSuccess)
    e = mg::launch_me_gluonhel(ctx->K, false, false, mom, nullptr, nevt, ctx->d_tab, ctx->d_gslots, 1 << ctx->K,
                               ctx->d_ngslots, ctx->d_mask, ctx->d_ctri, ctx->d_ctri_f, cst, ctx->d_part, stride,
                               ctx->side, nullptr, mg::MeShape(), nullptr, ctx->d_repair, ctx->d_nrepair, rows_out);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_join, ctx->side);
  return e;
}

static cudaError_t join_repair(mg_ctx* ctx, cudaStream_t st) { return cudaStreamWaitEvent(st, ctx->ev_join, 0); }

mg_status mg_sigmakin(mg_ctx* ctx, const double* mom_dev, int64_t nevt, mg_precision precision, double* me_dev,
                      void* stream) {
  if (!ctx || nevt < 0 || (nevt > 0 && (!mom_dev || !me_dev))) return MG_EINVAL;
  if (precision != MG_FP64 && precision != MG_FP32_AMP && precision != MG_FP64_TCCOLOR && precision != MG_MIXED)
    return MG_EINVAL;
  const bool tc = precision == MG_FP64_TCCOLOR || precision == MG_MIXED;
  if (tc && ctx->prm.wt != 0.0) return MG_ENOTSUP;   // the tensor-core colour path has zero top width
  if (nevt == 0) return MG_OK;
  // FP32 amplitudes with the lane-group kernel: the tensor-core colour sum runs inside it (no jamps)
  const bool mixed_in_kernel = mg::mixed_in_kernel(ctx, precision);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!ctx->mask_ready) {
    mg_status s = mg_hel_filter(ctx, mom_dev, nevt, stream);
    if (s != MG_OK) return s;
  }
  const int64_t stride = pad32(nevt);
  mg_status s = grow(&ctx->d_part, &ctx->part_cap, stride * ctx->nhel);
  if (s != MG_OK) return s;
  ctx->last = st;
  const mg::MeConst cst = me_const(ctx);
  const double norm = 1.0 / (256.0 * mg::factorial(ctx->ng));
  if (tc && !mixed_in_kernel) {
    // amplitudes -> FP32 jamps -> tensor-core colour sums, in chunks of whole pages that keep the jamp
    // buffer within 4 GiB
    const bool fp32 = precision == MG_MIXED;
    const bool warp = fp32 && ctx->shape[precision].warp && mg::me_warp_available(ctx->K, true);
    const bool fused = fp32 && !warp && ctx->shape[precision].fused && ctx->shape[precision].unrolled &&
                       mg::me_static_available(ctx->K, true);
    const int64_t per_event = static_cast<int64_t>(ctx->nhel) * ctx->ncol;   // float2 per event
    int64_t chunk = (int64_t(1) << 29) / per_event;                          // 2^29 float2 = 4 GiB
    chunk = chunk / mg::kPage * mg::kPage;
    if (chunk < mg::kPage) chunk = mg::kPage;
    if (chunk > stride) chunk = stride;
    // FP64 amplitudes: optionally the currents shared between gluon-helicity combinations (as MG_FP64)
    const bool shared = !fp32 && ctx->shape[precision].shared;
    if (shared) {
      const int64_t sc = mg::share_chunk(ctx->K, stride);
      if (sc < chunk) chunk = sc;
      s = grow(&ctx->d_share, &ctx->share_cap, chunk * mg::share_doubles(ctx->K));
      if (s != MG_OK) return s;
    }
    if (ctx->jamp_cap < chunk * per_event) {
      if (ctx->d_jamps) mg::dev_free(ctx->d_jamps);
      ctx->d_jamps = nullptr;
      ctx->jamp_cap = 0;
      if (mg::dev_alloc(&ctx->d_jamps, static_cast<size_t>(chunk * per_event) * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        return MG_ENOMEM;
      }
      ctx->jamp_cap = chunk * per_event;
    }
    s = grow(&ctx->d_prep, &ctx->prep_cap, chunk * mg::event_record_bytes(ctx->K, fp32) / 8 + 1);
    if (s == MG_OK && fp32) s = grow_repair(ctx, chunk);
    if (s != MG_OK) return s;
    for (int64_t e0 = 0; e0 < nevt; e0 += chunk) {
      const int64_t n = nevt - e0 < chunk ? nevt - e0 : chunk;
      const int64_t cst_stride = pad32(n);
      const double* mom_c = mom_dev + (e0 / mg::kPage) * ctx->npar * 4 * mg::kPage;
      if (fp32) {
        MG_CUDA(cudaMemsetAsync(ctx->d_nrepair, 0, sizeof(int), st));
        MG_CUDA(mg::launch_event_flags(ctx->K, mom_c, n, cst, ctx->d_repair, ctx->d_nrepair, ctx->d_flag, st));
      }
      if (!fused) MG_CUDA(mg::launch_event_prep(ctx->K, fp32, mom_c, n, cst, ctx->d_prep, st));
      // events with a small internal invariant: double-float or FP64 amplitudes (row layout), on the
      // side stream while the FP32 launches, which skip them, run
      if (fp32) MG_CUDA(fork_repair(ctx, mom_c, n, cst, cst_stride, 1, ctx->shape[precision].df_redo, st));
      if (fused)
        MG_CUDA(mg::launch_me_fused(ctx->K, true, mom_c, n, ctx->d_gslots, ctx->d_ngslots, ctx->d_mask, cst, ctx->d_part,
                                    cst_stride, ctx->d_jamps, ctx->d_flag, st));
      else if (warp)
        MG_CUDA(mg::launch_me_warp(ctx->K, ctx->d_prep, n, ctx->d_tab, ctx->d_gslots, 1 << ctx->K, ctx->d_ngslots,
                                   ctx->d_mask, ctx->d_cfull, ctx->d_cmat, 1, cst, ctx->d_part, cst_stride, ctx->d_jamps,
                                   ctx->d_flag, st));
      else if (shared) {
        MG_CUDA(mg::launch_share(ctx->K, ctx->d_prep, n, ctx->d_tab, cst, ctx->d_share, st));
        MG_CUDA(mg::launch_me_gluonhel(ctx->K, false, false, mom_c, ctx->d_prep, n, ctx->d_tab, ctx->d_gslots, 1 << ctx->K,
                                       ctx->d_ngslots, ctx->d_mask, ctx->d_ctri, ctx->d_ctri_f, cst, ctx->d_part,
                                       cst_stride, st, ctx->d_jamps, ctx->shape[precision], nullptr, nullptr, nullptr, 0,
                                       ctx->d_share));
      }
      else
        MG_CUDA(mg::launch_me_gluonhel(ctx->K, fp32, false, mom_c, ctx->d_prep, n, ctx->d_tab, ctx->d_gslots, 1 << ctx->K,
                                       ctx->d_ngslots, ctx->d_mask, ctx->d_ctri, ctx->d_ctri_f, cst, ctx->d_part, cst_stride,
                                       st, ctx->d_jamps, ctx->shape[precision], fp32 ? ctx->d_flag : nullptr));
      if (ctx->shape[precision].tc_sync)
        MG_CUDA(mg::launch_colour_tc(ctx->ncol, ctx->d_jamps, n, ctx->nhel, ctx->d_nrows, ctx->d_cmat, cst.colour_scale,
                                     ctx->d_part, cst_stride, st, fp32 ? ctx->d_flag : nullptr));
      else
        MG_CUDA(mg::launch_colour_umma(ctx->ncol, ctx->d_jamps, n, ctx->nhel, ctx->d_nrows, ctx->d_cumma, cst.colour_scale,
                                       ctx->d_part, cst_stride, st, fp32 ? ctx->d_flag : nullptr, ctx->d_tcerr,
                                       ctx->tc_stall));
      if (fp32) MG_CUDA(join_repair(ctx, st));
      MG_CUDA(mg::launch_hel_sum(ctx->d_part, ctx->d_nrows, n, cst_stride, norm, me_dev + e0, st));
    }
  } else if (ctx->prm.wt == 0.0) {
    const bool fp32 = precision == MG_FP32_AMP || mixed_in_kernel;
    const bool warp = fp32 && ctx->shape[precision].warp && mg::me_warp_available(ctx->K, true);
    const bool fused = fp32 && !warp && ctx->shape[precision].fused && ctx->shape[precision].unrolled &&
                       mg::me_static_available(ctx->K, true);
    s = grow(&ctx->d_prep, &ctx->prep_cap, stride * mg::event_record_bytes(ctx->K, fp32) / 8 + 1);
    if (s == MG_OK && fp32) s = grow_repair(ctx, stride);
    if (s != MG_OK) return s;
    if (fp32) {
      MG_CUDA(cudaMemsetAsync(ctx->d_nrepair, 0, sizeof(int), st));
      MG_CUDA(mg::launch_event_flags(ctx->K, mom_dev, nevt, cst, ctx->d_repair, ctx->d_nrepair, ctx->d_flag, st));
    }
    if (!fused) MG_CUDA(mg::launch_event_prep(ctx->K, fp32, mom_dev, nevt, cst, ctx->d_prep, st));
    // events with a small internal invariant: recomputed with double-float or FP64 amplitudes (per-slot
    // layout) on the side stream
    if (fp32) MG_CUDA(fork_repair(ctx, mom_dev, nevt, cst, stride, 0, ctx->shape[precision].df_redo, st));
    const bool shared = !fp32 && ctx->shape[precision].shared;
    if (shared) {
      // FP64: the currents of fewer than all gluons once per helicity assignment of their gluons, then
      // the matrix elements reading them; in chunks of events that bound the scratch
      const int64_t chunk = mg::share_chunk(ctx->K, stride);
      s = grow(&ctx->d_share, &ctx->share_cap, chunk * mg::share_doubles(ctx->K));
      if (s != MG_OK) return s;
      const int64_t nitem = mg::event_record_bytes(ctx->K, false) / 8;
      for (int64_t e0 = 0; e0 < nevt; e0 += chunk) {
        const int64_t n = nevt - e0 < chunk ? nevt - e0 : chunk;
        const double* rec_c = ctx->d_prep + (e0 / mg::kPage) * nitem * mg::kPage;
        const double* mom_c = mom_dev + (e0 / mg::kPage) * ctx->npar * 4 * mg::kPage;
        MG_CUDA(mg::launch_share(ctx->K, rec_c, n, ctx->d_tab, cst, ctx->d_share, st));
        MG_CUDA(mg::launch_me_gluonhel(ctx->K, false, false, mom_c, const_cast<double*>(rec_c), n, ctx->d_tab,
                                       ctx->d_gslots, 1 << ctx->K, ctx->d_ngslots, ctx->d_mask, ctx->d_ctri,
                                       ctx->d_ctri_f, cst, ctx->d_part + e0, stride, st, nullptr, ctx->shape[precision],
                                       nullptr, nullptr, nullptr, 0, ctx->d_share));
      }
    } else if (fused)
      MG_CUDA(mg::launch_me_fused(ctx->K, true, mom_dev, nevt, ctx->d_gslots, ctx->d_ngslots, ctx->d_mask, cst,
                                  ctx->d_part, stride, nullptr, ctx->d_flag, st));
    else if (warp)
      MG_CUDA(mg::launch_me_warp(ctx->K, ctx->d_prep, nevt, ctx->d_tab, ctx->d_gslots, 1 << ctx->K, ctx->d_ngslots,
                                 ctx->d_mask, ctx->d_cfull, ctx->d_cmat, mixed_in_kernel ? 2 : 0, cst, ctx->d_part,
                                 stride, nullptr, ctx->d_flag, st));
    else
      MG_CUDA(mg::launch_me_gluonhel(ctx->K, fp32, false, mom_dev, ctx->d_prep, nevt, ctx->d_tab, ctx->d_gslots,
                                     1 << ctx->K, ctx->d_ngslots, ctx->d_mask, ctx->d_ctri, ctx->d_ctri_f, cst, ctx->d_part,
                                     stride, st, nullptr, ctx->shape[precision], fp32 ? ctx->d_flag : nullptr));
    if (fp32) MG_CUDA(join_repair(ctx, st));
    MG_CUDA(mg::launch_hel_sum(ctx->d_part, ctx->d_ngslots, nevt, stride, norm, me_dev, st));
  } else {
    MG_CUDA(mg::launch_me_helicity(ctx->K, precision == MG_FP32_AMP, mom_dev, nevt, ctx->d_tab, ctx->d_good, ctx->nhel,
                                   ctx->d_ngood, ctx->d_ctri, cst, ctx->d_part, stride, st));
    MG_CUDA(mg::launch_hel_sum(ctx->d_part, ctx->d_ngood, nevt, stride, norm, me_dev, st));
  }
  return MG_OK;
}

mg_status mg_sigmakin_host(mg_ctx* ctx, const double* mom_host, int64_t nevt, mg_precision precision,
                           double* me_host, void* stream) {
  if (!ctx || nevt < 0 || (nevt > 0 && (!mom_host || !me_host))) return MG_EINVAL;
  if (nevt == 0) return MG_OK;
  const int64_t nmom = mg_mom_count(ctx->proc, nevt);
  if (ctx->stage_cap < nmom + pad32(nevt)) {
    if (ctx->d_mom_stage) mg::dev_free(ctx->d_mom_stage);
    if (ctx->d_me_stage) mg::dev_free(ctx->d_me_stage);
    ctx->d_mom_stage = ctx->d_me_stage = nullptr;
    ctx->stage_cap = 0;
    if (mg::dev_alloc(&ctx->d_mom_stage, nmom * sizeof(double)) != cudaSuccess ||
        mg::dev_alloc(&ctx->d_me_stage, pad32(nevt) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return MG_ENOMEM;
    }
    ctx->stage_cap = nmom + pad32(nevt);
  }
  if (!ctx->cp_in) {
    if (cudaStreamCreateWithFlags(&ctx->cp_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->cp_out, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return MG_ECUDA;
    }
    for (int c = 0; c < mg_ctx::kHostChunks; ++c)
      if (cudaEventCreateWithFlags(&ctx->ev_in[c], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ctx->ev_done[c], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return MG_ECUDA;
      }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // up to kHostChunks chunks of whole 32-event pages, each of at least 16,384 events: the copies in run
  // on cp_in, the matrix elements of chunk c on st once its momenta are in, its results go out on cp_out.
  // Per-event results do not depend on the chunking (the helicity filter of a first call sees the same
  // first events, a chunk holding at least 16,384 of them).
  int64_t nch = nevt / 16384;
  if (nch < 1) nch = 1;
  if (nch > mg_ctx::kHostChunks) nch = mg_ctx::kHostChunks;
  const int64_t chunk = pad32((nevt + nch - 1) / nch);
  const int64_t per_page = static_cast<int64_t>(ctx->npar) * 4 * mg::kPage;
  int nc = 0;
  for (int64_t e0 = 0; e0 < nevt; e0 += chunk, ++nc) {
    const int64_t n = nevt - e0 < chunk ? nevt - e0 : chunk;
    const int64_t off = e0 / mg::kPage * per_page;
    MG_CUDA(cudaMemcpyAsync(ctx->d_mom_stage + off, mom_host + off, pad32(n) / mg::kPage * per_page * sizeof(double),
                            cudaMemcpyHostToDevice, ctx->cp_in));
    MG_CUDA(cudaEventRecord(ctx->ev_in[nc], ctx->cp_in));
  }
  nc = 0;
  for (int64_t e0 = 0; e0 < nevt; e0 += chunk, ++nc) {
    const int64_t n = nevt - e0 < chunk ? nevt - e0 : chunk;
    const int64_t off = e0 / mg::kPage * per_page;
    MG_CUDA(cudaStreamWaitEvent(st, ctx->ev_in[nc], 0));
    mg_status s = mg_sigmakin(ctx, ctx->d_mom_stage + off, n, precision, ctx->d_me_stage + e0, stream);
    if (s != MG_OK) {
      cudaStreamSynchronize(ctx->cp_in);
      cudaStreamSynchronize(ctx->cp_out);
      return s;
    }
    MG_CUDA(cudaEventRecord(ctx->ev_done[nc], st));
    MG_CUDA(cudaStreamWaitEvent(ctx->cp_out, ctx->ev_done[nc], 0));
    MG_CUDA(cudaMemcpyAsync(me_host + e0, ctx->d_me_stage + e0, n * sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->cp_out));
  }
  MG_CUDA(cudaStreamSynchronize(ctx->cp_out));
  return MG_OK;
}

mg_status mg_hel_mask(mg_ctx* ctx, uint32_t* mask_host, int* ngood) {
  if (!ctx || !mask_host || !ngood) return MG_EINVAL;
  MG_CUDA(cudaStreamSynchronize(ctx->last));
  const int nw = (ctx->nhel + 31) / 32;
  MG_CUDA(cudaMemcpy(mask_host, ctx->d_mask, nw * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  MG_CUDA(cudaMemcpy(ngood, ctx->d_ngood, sizeof(int), cudaMemcpyDeviceToHost));
  return MG_OK;
}

mg_status mg_check(mg_ctx* ctx, void* stream, int64_t* nbad) {
  if (!ctx) return MG_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) { cudaGetLastError(); return MG_ECUDA; }
  unsigned long long n = 0;
  int tcerr = 0;
  MG_CUDA(cudaMemcpy(&n, ctx->d_nbad, sizeof(n), cudaMemcpyDeviceToHost));
  MG_CUDA(cudaMemset(ctx->d_nbad, 0, sizeof(n)));
  MG_CUDA(cudaMemcpy(&tcerr, ctx->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost));
  MG_CUDA(cudaMemset(ctx->d_tcerr, 0, sizeof(int)));
  if (nbad) *nbad = static_cast<int64_t>(n);
  if (tcerr) return MG_ETIMEOUT;
  return n ? MG_ENOCONV : MG_OK;
}

int64_t mg_kernel_launches(void) { return mg::g_launches.load(std::memory_order_relaxed); }

mg_status mg_diag_fail_alloc(int64_t nth) {
  if (nth < 0) return MG_EINVAL;
  mg::g_fail_countdown.store(nth);
  return MG_OK;
}

int64_t mg_diag_live_allocs(void) { return mg::g_live_allocs.load(); }

mg_status mg_diag_tc_stall(mg_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return MG_EINVAL;
  ctx->tc_stall = on;
  return MG_OK;
}

}  // extern "C"
