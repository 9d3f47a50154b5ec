// mg_kernels.h -- launch wrappers of the engine's device kernels (host-callable).
#pragma once

#include <cuda_runtime.h>

#include "mg_internal.h"

namespace mg {

constexpr int kMeThreads = 128;

struct MeConst {
  double gs;            // strong coupling g_s = sqrt(4 pi alpha_s)
  double mt, wt;        // top mass and width
  double colour_scale;  // g_s^2 / colour-matrix denominator
  double fp32_tau = 3e-4;  // FP32 modes: events with an internal invariant below fp32_tau * s are redone in FP64
};

// Launch shape of the matrix-element kernel: a block of kMeThreads threads covers tile_ev events x
// (kMeThreads / tile_ev) gluon-helicity slots (tile_ev in {32, 64, 128}); slot_major orders the grid so
// that all slot tiles of an event tile are dispatched together (the event's per-event record is then
// re-read from L2), else all event tiles of a slot tile come first.
// unrolled: use the kernel with the recursion expanded at compile time (mg_me3.cu) where it exists
// (me_static_available), else the one that reads the recursion tables at run time (mg_me2.cu).
// df_redo: the FP32 modes recompute their flagged events with double-float (else FP64) amplitudes.
// fused: (unrolled FP32 kernel only) the per-event record is computed inside the matrix-element kernel
// (k_me_fused: 32 events per block, the slots looped by its warps; tile_ev and slot_major unused).
// warp: (FP32, where me_warp_available) one lane group per (event, slot), state in shared memory
// (mg_me_warp.cu); takes precedence over unrolled.  tc_apart: MG_MIXED with warp writes the jamps out for
// launch_colour_tc instead of summing the colours on the tensor cores in the kernel.
struct MeShape {
  int tile_ev = 128;
  bool slot_major = false;
  bool unrolled = true;
  bool df_redo = true;
  bool fused = true;
  bool warp = false;
  bool tc_apart = false;
  bool shared = true;   // FP64 amplitudes: currents of fewer than all gluons shared between slots
  bool tc_sync = false;  // separate colour pass on mma.sync (k_colour_tc) instead of tcgen05 (k_colour_umma)
};

cudaError_t launch_philox(uint64_t seed, int64_t nevt, int nfinal, uint32_t* words, cudaStream_t st);
cudaError_t launch_rambo(int K, uint64_t seed, int64_t e0, int64_t nevt, double sqrts, double mt, double w0,
                         double* mom, double* wgt, unsigned long long* nbad, cudaStream_t st);
// out[slot * stride + e] = colour-summed |M_h|^2 of event e for helicity hels[slot]
// (slots >= *nslot exit at once, so the helicity count can stay on the device)
cudaError_t launch_me_helicity(int K, bool fp32, const double* mom, int64_t nevt, const Tables* tab, const int* hels,
                               int maxslot, const int* nslot, const double* ctri, const MeConst& cst, double* out,
                               int64_t stride, cudaStream_t st);
// Per-event record (momenta sums, propagator factors, wavefunctions; FP64 arithmetic, stored as FP32 or
// FP64) of every event into rec (ceil(nevt/32)*32 * event_record_bytes(K, fp32) bytes).
cudaError_t launch_event_prep(int K, bool fp32, const double* mom, int64_t nevt, const MeConst& cst, void* rec,
                              cudaStream_t st);
// FP32 modes: flag[e] = 1 and e appended to repair[] (count *nrepair, zero before the launch) for the events
// whose smallest internal invariant is below cst.fp32_tau * s; flag[e] = 0 for the others.
cudaError_t launch_event_flags(int K, const double* mom, int64_t nevt, const MeConst& cst, int* repair, int* nrepair,
                               uint8_t* flag, cudaStream_t st);
// One thread per (event, gluon-helicity combination gslots[slot]); per_hel: out[h * stride + e] for every
// helicity h of the combination, else out[slot * stride + e] = sum over its good helicities.  Zero top width.
// prep: NULL (every thread computes its event's momenta sums, propagators and wavefunctions) or the
// records launch_event_prep wrote; with prep, events with skip[e] != 0 (skip optional) are left out
// (nothing written).  evlist/nlist (prep == NULL only): work on events evlist[0..*nlist) of the batch;
// rows_out: write slot totals in the tensor-core row layout (4 rows per slot).
cudaError_t launch_me_gluonhel(int K, bool fp32, bool per_hel, const double* mom, void* prep, int64_t nevt,
                               const Tables* tab, const int* gslots, int maxslot, const int* nslot,
                               const uint32_t* mask, const double* ctri64, const float* ctri32, const MeConst& cst,
                               double* out, int64_t stride, cudaStream_t st, float2* jout = nullptr,
                               MeShape shape = MeShape(), const uint8_t* skip = nullptr,
                               const int* evlist = nullptr, const int* nlist = nullptr, int rows_out = 0,
                               const double* share = nullptr);
// FP64 currents shared between gluon-helicity combinations: share_items(K) items of 24 doubles per event
// (layout in mg_me_kernel.cuh), computed from the FP64 records of nevt events by K - 1 launches (one per
// sequence length); launch_me_gluonhel(..., share) then reads them instead of computing them per slot.
int share_items(int K);
// doubles per event of the shared buffer: the current items, then the quark-line prefixes (mg_internal.h)
int64_t share_doubles(int K);
cudaError_t launch_share(int K, const void* rec, int64_t nevt, const Tables* tab, const MeConst& cst, double* share,
                         cudaStream_t st);
int64_t event_record_bytes(int K, bool fp32);
// The FP32 modes' recomputation of events evlist[0..*nlist) with double-float amplitudes (mg_me_dd.cu):
// launch_me_gluonhel's contract for prep == NULL, per_hel false, FP32 colour table ctri32 (the per-thread
// kernel) or full FP32 colour matrix cfull (the lane-group kernel, used for 4 and 5 gluons).
cudaError_t launch_me_repair(int K, const double* mom, int64_t nevt, const Tables* tab, const int* gslots, int maxslot,
                             const int* nslot, const uint32_t* mask, const float* ctri32, const float* cfull,
                             const MeConst& cst, double* out, int64_t stride, const int* evlist, const int* nlist,
                             int rows_out, cudaStream_t st);
// The lane-group form of that recomputation (mg_me_warp.cu, K = 3..5).
cudaError_t launch_me_warp_repair(int K, const double* mom, int64_t nevt, const Tables* tab, const int* gslots,
                                  int maxslot, const int* nslot, const uint32_t* mask, const float* cfull,
                                  const MeConst& cst, double* out, int64_t stride, const int* evlist, const int* nlist,
                                  int rows_out, cudaStream_t st);
// The compile-time-unrolled matrix-element kernel (mg_me3.cu): same contract as launch_me_gluonhel with
// a per-event record rec (filled by k_event_prep), for the (K, precision) pairs me_static_available
// lists.  me_static_upload_colour: its colour triangle (constant memory), once per device and K.
bool me_static_available(int K, bool fp32);
cudaError_t me_static_upload_colour(int K, const double* tri, int n);
cudaError_t launch_me_static(int K, bool fp32, const void* rec, int64_t nevt, const int* gslots, int maxslot,
                             const int* nslot, const uint32_t* mask, const MeConst& cst, double* out, int64_t stride,
                             float2* jout, MeShape shape, const uint8_t* skip, cudaStream_t st);
// The lane-group-per-(event, slot) FP32 kernel (mg_me_warp.cu): launch_me_gluonhel's contract with a record
// rec (FP32) from launch_event_prep.  epi 0: colour sums in FP32 with cfull (the full ncol x ncol numerator
// matrix in FP32); 1: jamps to jout for launch_colour_tc; 2: colour sums on the tensor cores in the kernel
// with cmat16 (the FP16 operand of launch_colour_tc).  Epilogues 0 and 2 write out[slot * stride + e].
bool me_warp_available(int K, bool fp32);
cudaError_t launch_me_warp(int K, const void* rec, int64_t nevt, const Tables* tab, const int* gslots, int maxslot,
                           const int* nslot, const uint32_t* mask, const float* cfull, const void* cmat16, int epi,
                           const MeConst& cst, double* out, int64_t stride, float2* jout, const uint8_t* skip,
                           cudaStream_t st);
// The same with the record computed inside the kernel from the momenta (no per-event kernel first).
cudaError_t launch_me_fused(int K, bool fp32, const double* mom, int64_t nevt, const int* gslots, const int* nslot,
                            const uint32_t* mask, const MeConst& cst, double* out, int64_t stride, float2* jout,
                            const uint8_t* skip, cudaStream_t st);

// Tensor-core colour sum (mg_colour_tc.cu): out[r * stride + e] = scale * (Re A^T C Re A + Im A^T C Im A)
// for the jamp rows jamps[(e * rows_alloc + r) * ncol ...], r < *nrows; events with skip[e] != 0 (skip
// optional) are not written.
int colour_tc_cmat_halves(int ncol);
// The separate tensor-core colour pass on the fifth-generation tensor cores (tcgen05.mma, accumulators in
// tensor memory): same rows, outputs and skip list as launch_colour_tc; cumma = colour_umma_pack's operand;
// a bounded wait that gives up leaves a nonzero stage code in *err (read by mg_check).
int colour_umma_halves(int ncol);
void colour_umma_pack(int ncol, const int64_t* num, uint16_t* out_halves);
cudaError_t launch_colour_umma(int ncol, const float2* jamps, int64_t nevt, int rows_alloc, const int* nrows,
                               const void* cumma, double scale, double* out, int64_t stride, cudaStream_t st,
                               const uint8_t* skip, int* err, int stall = 0);
void colour_tc_pack(int ncol, const int64_t* num, uint16_t* out_halves);
cudaError_t launch_colour_tc(int ncol, const float2* jamps, int64_t nevt, int rows_alloc, const int* nrows,
                             const void* cmat, double scale, double* out, int64_t stride, cudaStream_t st,
                             const uint8_t* skip = nullptr);
cudaError_t launch_gluon_slots(const uint32_t* mask, int K, int* gslots, int* n, int* nrows, cudaStream_t st);
cudaError_t launch_hel_sum(const double* part, const int* nslot, int64_t nevt, int64_t stride, double norm,
                           double* me, cudaStream_t st);
cudaError_t launch_hel_mask(const double* part, const double* tot, int nhel, int64_t nevt, int64_t stride, double tau,
                            double* maxr, uint32_t* mask, int* good, int* ngood, cudaStream_t st);

}  // namespace mg
