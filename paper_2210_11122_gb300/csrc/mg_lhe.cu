// mg_lhe.cu -- event-level epilogues of the FP64 matrix elements: per-event helicity and leading-colour
// choices for unweighted-event (LHE) files, and the running of the strong coupling.
//
// The paper (Sec. 4) names event-by-event helicities and leading colours as the two pieces missing from
// the LHE files written with its GPU matrix elements, and the running of alpha_s (Sec. 2) as a feature
// the engine gained; both are cheap per-event epilogues on quantities the matrix-element kernel already
// has: the colour-summed |M_h|^2 of every helicity and the colour-ordered amplitudes (jamps).
//   * helicity choice: the smallest good helicity h (ascending index) whose running sum of |M_h|^2
//     exceeds r_hel times the sum over all good helicities;
//   * colour choice: the smallest colour flow sigma (lexicographic permutation rank) whose running sum
//     of w_sigma = sum over good helicities of |J_sigma(h)|^2 exceeds r_col times the sum over sigma;
//   * running alpha_s: one-loop, alpha_s(mu) = alpha_s(M_Z) / (1 + alpha_s(M_Z) b0 ln(mu^2 / M_Z^2)),
//     b0 = (33 - 2 n_f) / (12 pi), n_f = 5, M_Z = 91.1876 GeV, at mu = H_T / 2 (half the sum of the
//     final-state transverse masses); every tree diagram of g g -> t tbar + n g carries g_s^(n+2), so the
//     matrix element at alpha_s(mu) is the one at the context's alpha_s times (alpha_s(mu)/alpha_s)^(n+2).
#include <cuda_runtime.h>

#include <cmath>

#include "mg_alloc.h"
#include "mg_ctx.h"
#include "mg_internal.h"
#include "mg_kernels.h"
#include "mg_me_kernel.cuh"

namespace mg {
namespace lhe {

constexpr double kMZ = 91.1876;
constexpr int kNf = 5;

// H_T / 2 of an event: half the sum of sqrt(m^2 + px^2 + py^2) over the final-state particles (t, tbar,
// final-state gluons), read from the AoSoA momenta.
template <int K>
__device__ __forceinline__ double half_ht(const double* __restrict__ mom, int64_t e, double mt) {
  constexpr int npar = K + 2;
  const double* base = mom + (e / kPage) * npar * 4 * kPage + (e % kPage);
  double ht = 0.0;
  for (int i = 2; i < npar; ++i) {
    const double px = base[(i * 4 + 1) * kPage], py = base[(i * 4 + 2) * kPage];
    const double m = i < 4 ? mt : 0.0;
    ht += sqrt(m * m + px * px + py * py);
  }
  return 0.5 * ht;
}

// One-loop alpha_s at mu from alpha_s(M_Z) = a0.
__device__ __forceinline__ double alphas_1loop(double a0, double mu) {
  const double b0 = (33.0 - 2.0 * kNf) / (12.0 * 3.14159265358979323846);
  return a0 / (1.0 + a0 * b0 * log(mu * mu / (kMZ * kMZ)));
}

// (alpha_s(mu) / a0)^K by repeated multiplication (K <= 5).
template <int K>
__device__ __forceinline__ double coupling_factor(double a0, double mu, double* as) {
  const double a = alphas_1loop(a0, mu);
  if (as) *as = a;
  const double r = a / a0;
  double f = r;
#pragma unroll
  for (int k = 1; k < K; ++k) f *= r;
  return f;
}

// One thread per event: helicity sum (ascending helicity index), helicity and colour choices, coupling.
// part rows: slot * 4 + 2 top + antitop (k_me_gluonhel<..., LHE>); j2: per-slot jamp-square sums.
template <int K>
__global__ void __launch_bounds__(128)
k_lhe_epilogue(const double* __restrict__ part, const double* __restrict__ j2, const int* __restrict__ gslots,
               const int* __restrict__ nslot_dev, const uint32_t* __restrict__ mask, const double* __restrict__ mom,
               int64_t nevt, int64_t stride, double norm, int running, double a0, double mt,
               const double* __restrict__ rnd_hel, const double* __restrict__ rnd_col, double* __restrict__ me_out,
               int* __restrict__ hel_out, int* __restrict__ col_out, double* __restrict__ as_out) {
  constexpr int npar = K + 2, NHEL = 1 << npar, NCOL = v2::Sizes<K>::ncol;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= nevt) return;
  const int nslot = *nslot_dev;
  int slot_of[1 << K];
#pragma unroll
  for (int g = 0; g < (1 << K); ++g) slot_of[g] = -1;
  for (int s = 0; s < nslot; ++s) slot_of[gslots[s]] = s;
  auto row_of = [&](int h) -> int {
    int gc = 0;
#pragma unroll
    for (int g = 0; g < K; ++g) gc |= ((h >> (npar - 1 - (g < 2 ? g : g + 2))) & 1) << g;
    const int a = (h >> (npar - 3)) & 1, b = (h >> (npar - 4)) & 1;
    return slot_of[gc] * 4 + 2 * a + b;
  };
  auto good = [&](int h) -> bool { return (mask[h >> 5] >> (h & 31)) & 1u; };
  double total = 0.0;
  int last = -1;
  for (int h = 0; h < NHEL; ++h)
    if (good(h)) {
      total += part[row_of(h) * stride + e];
      last = h;
    }
  double f = 1.0, as = a0;
  if (running) f = coupling_factor<K>(a0, half_ht<K>(mom, e, mt), &as);
  me_out[e] = total * norm * f;
  if (as_out) as_out[e] = as;
  if (hel_out) {
    const double target = rnd_hel[e] * total;
    double cum = 0.0;
    int pick = last;
    for (int h = 0; h < NHEL; ++h)
      if (good(h)) {
        cum += part[row_of(h) * stride + e];
        if (cum > target) { pick = h; break; }
      }
    hel_out[e] = pick;
  }
  if (col_out) {
    double w[NCOL];
    double totc = 0.0;
    for (int c = 0; c < NCOL; ++c) {
      double acc = 0.0;
      for (int s = 0; s < nslot; ++s) acc += j2[(static_cast<int64_t>(s) * NCOL + c) * stride + e];
      w[c] = acc;
      totc += acc;
    }
    const double target = rnd_col[e] * totc;
    double cum = 0.0;
    int pick = NCOL - 1;
    for (int c = 0; c < NCOL; ++c) {
      cum += w[c];
      if (cum > target) { pick = c; break; }
    }
    col_out[e] = pick;
  }
}

// Coupling only, for the matrix elements of any precision mode: me[e] *= (alpha_s(mu_e)/a0)^K.
template <int K>
__global__ void __launch_bounds__(128)
k_alphas_running(const double* __restrict__ mom, int64_t nevt, double a0, double mt, double* __restrict__ me,
                 double* __restrict__ as_out) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= nevt) return;
  double as;
  const double f = coupling_factor<K>(a0, half_ht<K>(mom, e, mt), &as);
  me[e] *= f;
  if (as_out) as_out[e] = as;
}

// The slot kernel's LHE rows with the currents and quark-line prefixes of launch_share, compiled for
// MINB resident blocks per SM (the bound of the plain FP64 slot kernel)
template <int K, int MINB>
__global__ void __launch_bounds__(kMeThreads, MINB)
k_lhe_slot(const double* __restrict__ rec, int64_t nevt, const Tables* __restrict__ tab, const int* __restrict__ gslots,
           const int* __restrict__ nslot, const uint32_t* __restrict__ mask, const double* __restrict__ ctri, MeConst cst,
           double* __restrict__ part, int64_t stride, int tile_ev, const double* __restrict__ share,
           double* __restrict__ j2) {
  v2::me_thread<K, double, false, true, false, true, true>(nullptr, rec, nevt, tab, gslots, nslot, mask, ctri, cst, part,
                                                          stride, nullptr, tile_ev, 0, nullptr, nullptr, 0, nullptr,
                                                          share, j2);
}

// share: the chunk's currents and quark-line prefixes from launch_share (the slot kernel reads them
// instead of forming them; bit-identical), or null for the unshared walk
template <int K>
cudaError_t launch_lhe_me(const double* rec, int64_t nevt, const Tables* tab, const int* gslots, int maxslot,
                          const int* nslot, const uint32_t* mask, const double* ctri, const MeConst& cst, double* part,
                          double* j2, int64_t stride, const double* share, cudaStream_t st) {
  const int tev = 128, tsl = kMeThreads / tev;
  const dim3 grid(static_cast<unsigned>((nevt + tev - 1) / tev), static_cast<unsigned>((maxslot + tsl - 1) / tsl));
  // bounded compile for 2, 3 and 5 gluons (measured 12-25 % faster than unbounded); with 4 its 24 per-flow
  // sums spill at 168 registers and the unbounded kernel is 7 % faster
  if (share) {
    if constexpr (K == 4)
      v2::k_me_gluonhel<K, double, false, true, false, true, true><<<grid, kMeThreads, 0, st>>>(
          nullptr, rec, nevt, tab, gslots, nslot, mask, ctri, cst, part, stride, nullptr, tev, 0, nullptr, nullptr, 0,
          nullptr, share, j2);
    else
      k_lhe_slot<K, K <= 3 ? 4 : 3><<<grid, kMeThreads, 0, st>>>(rec, nevt, tab, gslots, nslot, mask, ctri, cst, part,
                                                                stride, tev, share, j2);
  } else
    v2::k_me_gluonhel<K, double, false, true, false, false, true><<<grid, kMeThreads, 0, st>>>(
        nullptr, rec, nevt, tab, gslots, nslot, mask, ctri, cst, part, stride, nullptr, tev, 0, nullptr, nullptr, 0,
        nullptr, nullptr, j2);
  note_launch();
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_epilogue(const double* part, const double* j2, const int* gslots, const int* nslot,
                            const uint32_t* mask, const double* mom, int64_t nevt, int64_t stride, double norm,
                            int running, double a0, double mt, const double* rnd_hel, const double* rnd_col,
                            double* me, int* hel, int* col, double* as, cudaStream_t st) {
  k_lhe_epilogue<K><<<static_cast<unsigned>((nevt + 127) / 128), 128, 0, st>>>(
      part, j2, gslots, nslot, mask, mom, nevt, stride, norm, running, a0, mt, rnd_hel, rnd_col, me, hel, col, as);
  note_launch();
  return cudaGetLastError();
}

}  // namespace lhe
}  // namespace mg

namespace {

int64_t pad_page(int64_t n) { return (n + mg::kPage - 1) / mg::kPage * mg::kPage; }

mg_status grow_buf(double** buf, int64_t* cap, int64_t need) {
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

cudaError_t lhe_me(int K, const double* rec, int64_t nevt, const mg_ctx* c, const mg::MeConst& cst, double* part,
                   double* j2, int64_t stride, const double* share, cudaStream_t st) {
  const int ms = 1 << K;
  switch (K) {
    case 2: return mg::lhe::launch_lhe_me<2>(rec, nevt, c->d_tab, c->d_gslots, ms, c->d_ngslots, c->d_mask, c->d_ctri, cst, part, j2, stride, share, st);
    case 3: return mg::lhe::launch_lhe_me<3>(rec, nevt, c->d_tab, c->d_gslots, ms, c->d_ngslots, c->d_mask, c->d_ctri, cst, part, j2, stride, share, st);
    case 4: return mg::lhe::launch_lhe_me<4>(rec, nevt, c->d_tab, c->d_gslots, ms, c->d_ngslots, c->d_mask, c->d_ctri, cst, part, j2, stride, share, st);
    case 5: return mg::lhe::launch_lhe_me<5>(rec, nevt, c->d_tab, c->d_gslots, ms, c->d_ngslots, c->d_mask, c->d_ctri, cst, part, j2, stride, share, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t lhe_epilogue(int K, const double* j2, const mg_ctx* c, const double* mom, int64_t nevt, int64_t stride,
                         double norm, int running, const double* rh, const double* rc, double* me, int* hel, int* col,
                         double* as, cudaStream_t st) {
  const double a0 = c->prm.alphas, mt = c->prm.mt;
  switch (K) {
    case 2: return mg::lhe::launch_epilogue<2>(c->d_part, j2, c->d_gslots, c->d_ngslots, c->d_mask, mom, nevt, stride, norm, running, a0, mt, rh, rc, me, hel, col, as, st);
    case 3: return mg::lhe::launch_epilogue<3>(c->d_part, j2, c->d_gslots, c->d_ngslots, c->d_mask, mom, nevt, stride, norm, running, a0, mt, rh, rc, me, hel, col, as, st);
    case 4: return mg::lhe::launch_epilogue<4>(c->d_part, j2, c->d_gslots, c->d_ngslots, c->d_mask, mom, nevt, stride, norm, running, a0, mt, rh, rc, me, hel, col, as, st);
    case 5: return mg::lhe::launch_epilogue<5>(c->d_part, j2, c->d_gslots, c->d_ngslots, c->d_mask, mom, nevt, stride, norm, running, a0, mt, rh, rc, me, hel, col, as, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

extern "C" {

mg_status mg_sigmakin_lhe(mg_ctx* ctx, const double* mom_dev, int64_t nevt, const double* rnd_hel_dev,
                          const double* rnd_col_dev, int running_alphas, double* me_dev, int* hel_dev, int* col_dev,
                          double* alphas_dev, void* stream) {
  if (!ctx || nevt < 0 || (nevt > 0 && (!mom_dev || !me_dev))) return MG_EINVAL;
  if ((hel_dev && !rnd_hel_dev) || (col_dev && !rnd_col_dev)) return MG_EINVAL;
  if (running_alphas != 0 && running_alphas != 1) return MG_EINVAL;
  if (ctx->prm.wt != 0.0) return MG_ENOTSUP;   // the per-event record has zero top width
  if (nevt == 0) return MG_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!ctx->mask_ready) {
    mg_status s = mg_hel_filter(ctx, mom_dev, nevt, stream);
    if (s != MG_OK) return s;
  }
  ctx->last = st;
  const int K = ctx->K;
  // chunks of whole pages that keep the per-slot jamp-square sums within 2^27 doubles (1 GiB)
  const int64_t per_event = static_cast<int64_t>(1 << K) * ctx->ncol;
  int64_t chunk = (int64_t(1) << 27) / per_event / mg::kPage * mg::kPage;
  const int64_t stride_all = pad_page(nevt);
  if (chunk < mg::kPage) chunk = mg::kPage;
  if (chunk > stride_all) chunk = stride_all;
  // the FP64 launch shape's choice of shared currents and prefixes (chunks within their buffer)
  const bool shared = ctx->shape[MG_FP64].shared;
  if (shared) {
    const int64_t sc = mg::share_chunk(K, stride_all);
    if (sc < chunk) chunk = sc;
  }
  mg_status s = grow_buf(&ctx->d_part, &ctx->part_cap, chunk * ctx->nhel);
  if (s == MG_OK) s = grow_buf(&ctx->d_prep, &ctx->prep_cap, chunk * mg::event_record_bytes(K, false) / 8 + 1);
  if (s == MG_OK) s = grow_buf(&ctx->d_j2, &ctx->j2_cap, chunk * per_event);
  if (s == MG_OK && shared) s = grow_buf(&ctx->d_share, &ctx->share_cap, chunk * mg::share_doubles(K));
  if (s != MG_OK) return s;
  mg::MeConst cst;
  cst.gs = std::sqrt(4.0 * 3.14159265358979323846 * ctx->prm.alphas);
  cst.mt = ctx->prm.mt;
  cst.wt = ctx->prm.wt;
  cst.colour_scale = cst.gs * cst.gs / static_cast<double>(ctx->colour_den);
  const double norm = 1.0 / (256.0 * mg::factorial(ctx->ng));
  for (int64_t e0 = 0; e0 < nevt; e0 += chunk) {
    const int64_t n = nevt - e0 < chunk ? nevt - e0 : chunk;
    const int64_t stride = pad_page(n);
    const double* mom_c = mom_dev + (e0 / mg::kPage) * ctx->npar * 4 * mg::kPage;
    if (mg::launch_event_prep(K, false, mom_c, n, cst, ctx->d_prep, st) != cudaSuccess) return MG_ECUDA;
    if (shared && mg::launch_share(K, ctx->d_prep, n, ctx->d_tab, cst, ctx->d_share, st) != cudaSuccess) return MG_ECUDA;
    if (lhe_me(K, ctx->d_prep, n, ctx, cst, ctx->d_part, ctx->d_j2, stride, shared ? ctx->d_share : nullptr, st) !=
        cudaSuccess)
      return MG_ECUDA;
    if (lhe_epilogue(K, ctx->d_j2, ctx, mom_c, n, stride, norm, running_alphas, rnd_hel_dev ? rnd_hel_dev + e0 : nullptr,
                     rnd_col_dev ? rnd_col_dev + e0 : nullptr, me_dev + e0, hel_dev ? hel_dev + e0 : nullptr,
                     col_dev ? col_dev + e0 : nullptr, alphas_dev ? alphas_dev + e0 : nullptr, st) != cudaSuccess)
      return MG_ECUDA;
  }
  return MG_OK;
}

mg_status mg_alphas_running(mg_ctx* ctx, const double* mom_dev, int64_t nevt, double* me_dev, double* alphas_dev,
                            void* stream) {
  if (!ctx || nevt < 0 || (nevt > 0 && (!mom_dev || !me_dev))) return MG_EINVAL;
  if (nevt == 0) return MG_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ctx->last = st;
  const unsigned blocks = static_cast<unsigned>((nevt + 127) / 128);
  const double a0 = ctx->prm.alphas, mt = ctx->prm.mt;
  switch (ctx->K) {
    case 2: mg::lhe::k_alphas_running<2><<<blocks, 128, 0, st>>>(mom_dev, nevt, a0, mt, me_dev, alphas_dev); break;
    case 3: mg::lhe::k_alphas_running<3><<<blocks, 128, 0, st>>>(mom_dev, nevt, a0, mt, me_dev, alphas_dev); break;
    case 4: mg::lhe::k_alphas_running<4><<<blocks, 128, 0, st>>>(mom_dev, nevt, a0, mt, me_dev, alphas_dev); break;
    case 5: mg::lhe::k_alphas_running<5><<<blocks, 128, 0, st>>>(mom_dev, nevt, a0, mt, me_dev, alphas_dev); break;
    default: return MG_EINVAL;
  }
  mg::note_launch();
  return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ECUDA;
}

mg_status mg_colour_flow(mg_process proc, int flow, int* order) {
  if (proc < MG_GG_TT || proc > MG_GG_TTGGG || !order) return MG_EINVAL;
  const int K = mg::gluons_of(proc), ncol = mg::factorial(K);
  if (flow < 0 || flow >= ncol) return MG_EINVAL;
  // the flow-th permutation of (0 .. K-1) in lexicographic order (factorial number system)
  int pool[mg::kMaxGluons];
  for (int i = 0; i < K; ++i) pool[i] = i;
  int rest = flow, n = K;
  for (int i = 0; i < K; ++i) {
    const int f = mg::factorial(n - 1);
    const int q = rest / f;
    rest -= q * f;
    order[i] = pool[q];
    for (int j = q; j + 1 < n; ++j) pool[j] = pool[j + 1];
    --n;
  }
  return MG_OK;
}

}  // extern "C"
