// mg_sde.cu -- single-diagram-enhancement channel weights (the MadEvent phase-space channels the paper's
// Sec. 2 lists among the engine's features).
//
// For channel d, a Feynman diagram built from three-point vertices only, the weight of an event is
//     w_d = sum_h |A_d(h)|^2 / sum_d' sum_h |A_d'(h)|^2       (good helicities h),
// A_d the amplitude of the diagram alone, colour factor stripped: gluon trees attached along the quark
// line from the top to the antitop, Feynman-gauge three-gluon vertices in full (single diagrams carry
// no current conservation, so the simplified vertex of the recursion does not apply), quark and gluon
// propagators.  The recursion of the matrix-element kernels sums diagrams into shared currents and never
// forms one diagram alone, so this is a separate, table-driven FP64 kernel:
//   * host: every binary gluon tree over every gluon subset (3 / 9 / 37 / 225 for 2..5 gluons, children
//     before parents) and a depth-first walk over the ordered lists of trees that partition the gluons
//     (a "push" attaches a tree and propagates the spinor, a "leaf" closes a diagram with the antitop):
//     3 / 15 / 105 / 945 channels;
//   * device: one thread per (event, gluon-helicity combination) builds every tree current once (the
//     gluon helicities fixed) and walks the list for each top helicity, the spinor prefixes on a stack,
//     adding |A_d|^2 of each good helicity into per-channel sums; a second kernel adds the combinations
//     and normalises per event.
// Every vertex carries one power of g (the quark propagators and gluon propagators of the per-event
// record carry it), so g^(n_g+1) and the propagator signs are common to all channels and cancel in w_d.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "mg_alloc.h"
#include "mg_ctx.h"
#include "mg_internal.h"
#include "mg_kernels.h"
#include "mg_me_algebra.cuh"

namespace mg {
namespace sde {

constexpr int kMaxNode = 225, kMaxOp = 1655, kMaxCh = 945;

struct Tab {
  int K, nnode, nop, nch;
  int16_t node_l[kMaxNode], node_r[kMaxNode];   // children (internal nodes); node_l = -1 - g for leaf g
  uint8_t node_mask[kMaxNode];
  int16_t op_node[kMaxOp], op_ch[kMaxOp];       // op_ch >= 0: closes channel op_ch; -1: attaches and propagates
  uint8_t op_depth[kMaxOp], op_mask[kMaxOp];    // trees before this one; gluons attached including this tree
};

template <int K> struct Sz;
template <> struct Sz<2> { static constexpr int nnode = 3, nop = 5, nch = 3; };
template <> struct Sz<3> { static constexpr int nnode = 9, nop = 27, nch = 15; };
template <> struct Sz<4> { static constexpr int nnode = 37, nop = 187, nch = 105; };
template <> struct Sz<5> { static constexpr int nnode = 225, nop = 1655, nch = 945; };

// Host: the trees, the walk and the channel keys ("1|2", "(1,2)", ... as documented in mg.h).
struct Built {
  Tab tab;
  std::vector<std::string> keys;
};

void build(int K, Built& out) {
  Tab& t = out.tab;
  std::memset(&t, 0, sizeof(t));
  t.K = K;
  std::vector<std::vector<int>> trees(1 << K);
  std::vector<std::string> nkey;
  for (int g = 0; g < K; ++g) {
    t.node_l[t.nnode] = static_cast<int16_t>(-1 - g);
    t.node_r[t.nnode] = -1;
    t.node_mask[t.nnode] = static_cast<uint8_t>(1 << g);
    trees[1 << g].push_back(t.nnode++);
    nkey.push_back(std::to_string(g + 1));
  }
  for (int pc = 2; pc <= K; ++pc)
    for (int S = 1; S < (1 << K); ++S) {
      if (__builtin_popcount(S) != pc) continue;
      const int low = S & -S;
      for (int A = (S - 1) & S; A; A = (A - 1) & S) {   // the part holding the lowest gluon
        if (!(A & low)) continue;
        const int B = S ^ A;
        for (int ta : trees[A])
          for (int tb : trees[B]) {
            t.node_l[t.nnode] = static_cast<int16_t>(ta);
            t.node_r[t.nnode] = static_cast<int16_t>(tb);
            t.node_mask[t.nnode] = static_cast<uint8_t>(S);
            trees[S].push_back(t.nnode++);
            nkey.push_back("(" + nkey[ta] + "," + nkey[tb] + ")");
          }
      }
    }
  std::vector<std::string> prefix;
  std::function<void(int, int, int)> walk = [&](int rem, int depth, int attached) {
    for (int S = rem; S; S = (S - 1) & rem)
      for (int n : trees[S]) {
        const int i = t.nop++;
        t.op_node[i] = static_cast<int16_t>(n);
        t.op_depth[i] = static_cast<uint8_t>(depth);
        t.op_mask[i] = static_cast<uint8_t>(attached | S);
        if (S == rem) {
          t.op_ch[i] = static_cast<int16_t>(t.nch++);
          std::string k;
          for (const std::string& p : prefix) k += p + "|";
          out.keys.push_back(k + nkey[n]);
        } else {
          t.op_ch[i] = -1;
          prefix.push_back(nkey[n]);
          walk(rem ^ S, depth + 1, attached | S);
          prefix.pop_back();
        }
      }
  };
  walk((1 << K) - 1, 0, 0);
}

const Built& built(int K) {
  static Built b[6];
  static std::once_flag once[6];
  std::call_once(once[K], [K] { build(K, b[K]); });
  return b[K];
}

using v2::cx;

// The three-gluon vertex in full, V = (JL.JR)(PL - PR) + (JL.(PL + 2 PR)) JR - (JR.(2 PL + PR)) JL
__device__ __forceinline__ void v3full(cx<double>* out, const cx<double>* JL, const cx<double>* JR, const double* PL,
                                       const double* PR, double f) {
  double a[4], b[4], d[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    d[m] = PL[m] - PR[m];
    a[m] = PL[m] + 2.0 * PR[m];
    b[m] = 2.0 * PL[m] + PR[m];
  }
  const cx<double> jj = v2::mdot(JL, JR), cl = v2::mdotr(JL, a), cr = v2::mdotr(JR, b);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    cx<double> acc = v2::cscale(d[m], jj);
    v2::cmac(acc, cl, JR[m]);
    v2::cmsub(acc, cr, JL[m]);
    out[m] = v2::cscale(f, acc);
  }
}

// One thread per (event, slot): per-channel sums of |A_d|^2 over the slot's good helicities into
// part[(slot * nch + d) * stride + e].
template <int K>
__global__ void __launch_bounds__(128) k_sde(const double* __restrict__ rec, int64_t nevt, const Tab* __restrict__ tab,
                                             const int* __restrict__ gslots, const int* __restrict__ nslot_dev,
                                             const uint32_t* __restrict__ mask, double* __restrict__ part,
                                             int64_t stride) {
  constexpr int npar = K + 2, NSUB = 1 << K, NN = Sz<K>::nnode, NOP = Sz<K>::nop, NCH = Sz<K>::nch;
  using L = v2::EvLayout<K>;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int slot = blockIdx.y;
  if (e >= nevt || slot >= *nslot_dev) return;
  const int gc = gslots[slot];
  const double* in = rec + (e / kPage) * L::NITEM * kPage + (e % kPage);
  auto ld = [&](int item) -> double { return __ldg(in + item * kPage); };
  double PT[NSUB][4], gprop[NSUB], qc[NSUB][5];
  for (int S = 1; S < NSUB; ++S) {
#pragma unroll
    for (int m = 0; m < 4; ++m) PT[S][m] = S == NSUB - 1 ? 0.0 : ld(L::PT + 4 * S + m);   // (no tree has the full set as a child)
    gprop[S] = ld(L::GP + S);
#pragma unroll
    for (int c = 0; c < 5; ++c) qc[S][c] = S == NSUB - 1 ? 0.0 : ld(L::QC + 5 * S + c);
  }
  cx<double> ub[2][4], vv[2][4];
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      ub[l][a] = {ld(L::UB + (l * 4 + a) * 2), ld(L::UB + (l * 4 + a) * 2 + 1)};
      vv[l][a] = {ld(L::VV + (l * 4 + a) * 2), ld(L::VV + (l * 4 + a) * 2 + 1)};
    }
  // every tree current of the gluon helicities gc
  cx<double> J[NN][4];
  for (int n = 0; n < NN; ++n) {
    const int l = tab->node_l[n];
    if (l < 0) {
      const int g = -1 - l;
      double pol[5];
#pragma unroll
      for (int i = 0; i < 5; ++i) pol[i] = ld(L::EPS + 5 * g + i);
      v2::ext_gluon(pol, (gc >> g) & 1 ? 1 : -1, g >= 2, J[n]);
    } else {
      const int r = tab->node_r[n];
      const int S = tab->node_mask[n];
      v3full(J[n], J[l], J[r], PT[tab->node_mask[l]], PT[tab->node_mask[r]], gprop[S]);
    }
  }
  int hbase = 0;
#pragma unroll
  for (int g = 0; g < K; ++g)
    if ((gc >> g) & 1) hbase |= 1 << (npar - 1 - (g < 2 ? g : g + 2));
  double acc[NCH];
  for (int d = 0; d < NCH; ++d) acc[d] = 0.0;
  for (int a = 0; a < 2; ++a) {
    const int h0 = hbase | (a << (npar - 3)), h1 = h0 | (1 << (npar - 4));
    const bool good0 = (mask[h0 >> 5] >> (h0 & 31)) & 1u, good1 = (mask[h1 >> 5] >> (h1 & 31)) & 1u;
    if (!good0 && !good1) continue;
    cx<double> stk[K][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) stk[0][q] = ub[a][q];
    for (int i = 0; i < NOP; ++i) {
      const int n = tab->op_node[i], dep = tab->op_depth[i], ch = tab->op_ch[i];
      cx<double> t[4] = {};
      v2::row_gamma_acc(t, stk[dep], J[n], false);
      if (ch >= 0) {
        cx<double> a0 = {0.0, 0.0}, a1 = {0.0, 0.0};
        v2::sdot_acc(a0, t, vv[0], false);
        v2::sdot_acc(a1, t, vv[1], false);
        double s = 0.0;
        if (good0) s = fma(a0.r, a0.r, fma(a0.i, a0.i, s));
        if (good1) s = fma(a1.r, a1.r, fma(a1.i, a1.i, s));
        acc[ch] += s;
      } else {
        v2::row_prop(t, qc[tab->op_mask[i]], stk[dep + 1]);
      }
    }
  }
  for (int d = 0; d < NCH; ++d) part[(static_cast<int64_t>(slot) * NCH + d) * stride + e] = acc[d];
}

// One thread per event: w[d * ldw + e] = sum over slots of part / sum over channels and slots.
__global__ void __launch_bounds__(128) k_sde_norm(const double* __restrict__ part, int64_t nevt, int64_t stride,
                                                  int nch, const int* __restrict__ nslot_dev, double* __restrict__ w,
                                                  int64_t ldw) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= nevt) return;
  const int nslot = *nslot_dev;
  double tot = 0.0;
  for (int d = 0; d < nch; ++d) {
    double s = 0.0;
    for (int sl = 0; sl < nslot; ++sl) s += part[(static_cast<int64_t>(sl) * nch + d) * stride + e];
    w[d * ldw + e] = s;
    tot += s;
  }
  const double r = 1.0 / tot;
  for (int d = 0; d < nch; ++d) w[d * ldw + e] *= r;
}

}  // namespace sde
}  // namespace mg

namespace {

int64_t padp(int64_t n) { return (n + mg::kPage - 1) / mg::kPage * mg::kPage; }

mg_status growb(double** buf, int64_t* cap, int64_t need) {
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

template <int K>
cudaError_t launch_sde(const double* rec, int64_t n, const mg::sde::Tab* tab, const mg_ctx* c, double* part, int64_t stride,
                       cudaStream_t st) {
  const dim3 grid(static_cast<unsigned>((n + 127) / 128), static_cast<unsigned>(1 << K));
  mg::sde::k_sde<K><<<grid, 128, 0, st>>>(rec, n, tab, c->d_gslots, c->d_ngslots, c->d_mask, part, stride);
  mg::note_launch();
  return cudaGetLastError();
}

}  // namespace

extern "C" {

mg_status mg_sde_channels(mg_process proc, int* nchannels) {
  if (proc < MG_GG_TT || proc > MG_GG_TTGGG || !nchannels) return MG_EINVAL;
  *nchannels = mg::sde::built(mg::gluons_of(proc)).tab.nch;
  return MG_OK;
}

mg_status mg_sde_channel_key(mg_process proc, int channel, char* key, int keylen) {
  if (proc < MG_GG_TT || proc > MG_GG_TTGGG || !key || keylen < 1) return MG_EINVAL;
  const mg::sde::Built& b = mg::sde::built(mg::gluons_of(proc));
  if (channel < 0 || channel >= b.tab.nch) return MG_EINVAL;
  const std::string& k = b.keys[channel];
  if (static_cast<int>(k.size()) + 1 > keylen) return MG_EINVAL;
  std::memcpy(key, k.c_str(), k.size() + 1);
  return MG_OK;
}

mg_status mg_sde_weights(mg_ctx* ctx, const double* mom_dev, int64_t nevt, double* w_dev, void* stream) {
  if (!ctx || nevt < 0 || (nevt > 0 && (!mom_dev || !w_dev))) return MG_EINVAL;
  if (ctx->prm.wt != 0.0) return MG_ENOTSUP;   // the per-event record has zero top width
  if (nevt == 0) return MG_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!ctx->mask_ready) {
    mg_status s = mg_hel_filter(ctx, mom_dev, nevt, stream);
    if (s != MG_OK) return s;
  }
  const int K = ctx->K;
  const mg::sde::Built& b = mg::sde::built(K);
  if (!ctx->d_sdetab) {
    if (mg::dev_alloc(&ctx->d_sdetab, sizeof(mg::sde::Tab)) != cudaSuccess) { cudaGetLastError(); return MG_ENOMEM; }
    if (cudaMemcpy(ctx->d_sdetab, &b.tab, sizeof(mg::sde::Tab), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      return MG_ECUDA;
    }
  }
  ctx->last = st;
  // chunks of whole pages that keep the per-slot channel sums within 2^28 doubles (2 GiB)
  const int64_t per_event = static_cast<int64_t>(1 << K) * b.tab.nch;
  int64_t chunk = (int64_t(1) << 28) / per_event / mg::kPage * mg::kPage;
  if (chunk < mg::kPage) chunk = mg::kPage;
  if (chunk > padp(nevt)) chunk = padp(nevt);
  mg_status s = growb(&ctx->d_prep, &ctx->prep_cap, chunk * mg::event_record_bytes(K, false) / 8 + 1);
  if (s == MG_OK) s = growb(&ctx->d_sde, &ctx->sde_cap, chunk * per_event);
  if (s != MG_OK) return s;
  mg::MeConst cst;
  cst.gs = std::sqrt(4.0 * 3.14159265358979323846 * ctx->prm.alphas);
  cst.mt = ctx->prm.mt;
  cst.wt = ctx->prm.wt;
  cst.colour_scale = cst.gs * cst.gs / static_cast<double>(ctx->colour_den);
  const mg::sde::Tab* tab = static_cast<const mg::sde::Tab*>(ctx->d_sdetab);
  for (int64_t e0 = 0; e0 < nevt; e0 += chunk) {
    const int64_t n = nevt - e0 < chunk ? nevt - e0 : chunk;
    const int64_t stride = padp(n);
    const double* mom_c = mom_dev + (e0 / mg::kPage) * ctx->npar * 4 * mg::kPage;
    if (mg::launch_event_prep(K, false, mom_c, n, cst, ctx->d_prep, st) != cudaSuccess) return MG_ECUDA;
    cudaError_t e = cudaSuccess;
    switch (K) {
      case 2: e = launch_sde<2>(ctx->d_prep, n, tab, ctx, ctx->d_sde, stride, st); break;
      case 3: e = launch_sde<3>(ctx->d_prep, n, tab, ctx, ctx->d_sde, stride, st); break;
      case 4: e = launch_sde<4>(ctx->d_prep, n, tab, ctx, ctx->d_sde, stride, st); break;
      default: e = launch_sde<5>(ctx->d_prep, n, tab, ctx, ctx->d_sde, stride, st); break;
    }
    if (e != cudaSuccess) return MG_ECUDA;
    mg::sde::k_sde_norm<<<static_cast<unsigned>((n + 127) / 128), 128, 0, st>>>(ctx->d_sde, n, stride, b.tab.nch,
                                                                               ctx->d_ngslots, w_dev + e0, nevt);
    mg::note_launch();
    if (cudaGetLastError() != cudaSuccess) return MG_ECUDA;
  }
  return MG_OK;
}

}  // extern "C"
