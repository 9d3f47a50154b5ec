// mg_ctx.h -- layout of a context (struct mg_ctx of include/mg.h), shared by the engine's own
// translation units.
#pragma once

#include <cuda_runtime.h>

#include "mg_internal.h"
#include "mg_kernels.h"

struct mg_ctx {
  mg_process proc;
  int K, npar, nhel, ncol, ng;
  mg_params prm;
  mg::Tables* d_tab = nullptr;
  double* d_ctri = nullptr;   // packed upper triangle of the integer colour matrix, off-diagonal doubled
  float* d_ctri_f = nullptr;  // the same in FP32 (exact: integers < 2^24)
  float* d_cfull = nullptr;   // the full ncol x ncol numerator matrix in FP32 (warp-per-slot kernel)
  int64_t colour_den = 1;
  uint32_t* d_mask = nullptr;
  double* d_maxr = nullptr;   // per-helicity maximum ratio of the last helicity filter
  int* d_good = nullptr;      // good helicity list
  int* d_ngood = nullptr;
  int* d_allhel = nullptr;    // 0..nhel-1
  int* d_nhel = nullptr;      // nhel
  int* d_gslots = nullptr;    // gluon-helicity combinations with a good helicity
  int* d_ngslots = nullptr;
  int* d_nrows = nullptr;     // 4 * (number of gluon combinations): jamp rows per event
  void* d_cmat = nullptr;     // colour matrix numerators as the packed FP16 tensor-core operand
  void* d_cumma = nullptr;    // the same as the tcgen05 B operand (canonical no-swizzle K-major layout)
  int* d_tcerr = nullptr;     // nonzero: a bounded wait of the tcgen05 colour kernel gave up
  int tc_stall = 0;           // diagnostics (mg_diag_tc_stall): the tcgen05 colour kernel issues no MMAs
  unsigned long long* d_tiles = nullptr;   // mg_sigmakin_batch: tile counter of the persistent launch
  float2* d_jamps = nullptr;  // FP32 jamps of the tensor-core colour path
  int64_t jamp_cap = 0;       // in float2
  int* d_allg = nullptr;      // 0..2^K-1
  int* d_nallg = nullptr;     // 2^K
  unsigned long long* d_nbad = nullptr;
  double* d_part = nullptr;   // per-(helicity, event) colour sums
  int64_t part_cap = 0;
  double* d_tot = nullptr;    // per-event helicity sums of the filter
  double* d_prep = nullptr;   // per-event records (momenta sums, propagators, wavefunctions)
  int* d_repair = nullptr;    // FP32 modes: events recomputed in FP64, and their count
  int* d_nrepair = nullptr;
  uint8_t* d_flag = nullptr;  // FP32 modes: 1 for the events in d_repair (the FP32 launches skip them)
  int64_t repair_cap = 0;
  double* d_j2 = nullptr;      // mg_sigmakin_lhe: per-slot sums of |jamp|^2 over good helicities (one chunk)
  int64_t j2_cap = 0;         // in doubles
  void* d_sdetab = nullptr;    // mg_sde_weights: trees and walk of the channels (uploaded on first use)
  double* d_sde = nullptr;     // per-slot channel sums (one chunk of events)
  int64_t sde_cap = 0;         // in doubles
  double* d_share = nullptr;   // FP64: currents shared between gluon-helicity combinations (one chunk of events)
  int64_t share_cap = 0;      // in doubles
  cudaStream_t side = nullptr;         // FP32 modes: the FP64 recomputation runs here, beside the FP32 launches
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int64_t prep_cap = 0;       // in doubles
  int64_t tot_cap = 0;
  double* d_mom_stage = nullptr;
  double* d_me_stage = nullptr;
  int64_t stage_cap = 0;
  // mg_sigmakin_host: copy streams and per-chunk events (host->device copies of later chunks and
  // device->host copies of earlier ones overlap the matrix elements of the chunk in between)
  static constexpr int kHostChunks = 4;
  cudaStream_t cp_in = nullptr, cp_out = nullptr;
  cudaEvent_t ev_in[kHostChunks] = {}, ev_done[kHostChunks] = {};
  bool mask_ready = false;
  double fp32_tau = 3e-4;     // FP32 modes: events with an internal invariant below fp32_tau * s are recomputed
                              // (set per process at creation)
  mg::MeShape shape[4];       // launch shape of the matrix-element kernel per precision (autotuned)
  cudaStream_t last = nullptr;
};


namespace mg {
// events per chunk of the FP64 shared-current path (its scratch stays within 2 GiB)
int64_t share_chunk(int K, int64_t stride);
// MG_MIXED on the lane-group kernel: colour sums on the tensor cores inside it, per-slot outputs
bool mixed_in_kernel(const mg_ctx* ctx, mg_precision precision);
mg_status ctx_reserve(mg_ctx* ctx, int64_t nevt, mg_precision precision);
// Give dst (same process) the helicity mask of src: mask words, good-helicity and gluon-slot lists,
// stream-ordered on st (device-to-device copies), then dst->mask_ready.
mg_status ctx_copy_mask(mg_ctx* dst, const mg_ctx* src, cudaStream_t st);
int64_t footprint_bytes(mg_process proc, int64_t nevt, mg_precision precision);
}  // namespace mg
