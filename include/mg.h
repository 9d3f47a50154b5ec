/*
 * mg.h -- C ABI of the GB300 (sm_103a) engine for per-event tree-level QCD matrix elements of
 *         g g -> t tbar + n_g gluons, n_g = 0..3.
 *
 * The workflow follows arXiv 2210.11122 (Sec. 1, Fig. 1): random numbers -> phase-space
 * momenta -> matrix element (ME) per event, all on the GPU (the "standalone" application of
 * Sec. 1).  The ME is the per-event hot path of Sec. 2 (the paper's gg -> t tbar gg kernel uses
 * every one of the 255 registers of a thread) and its throughput is counted as
 * N_events / t_MEs (Sec. 2, Tables 1-2).  The paper prints no formulas; the physics below is the
 * textbook one (HELAS wavefunctions, Feynman-gauge QCD vertices, colour decomposition of
 * Mangano-Parke) with the conventions stated here.
 *
 * Conventions shared by every entry point
 *   - metric (+,-,-,-); momenta (E, px, py, pz) in GeV, FP64;
 *   - particle order g1, g2, t, tbar, g3, ..., g(2+n_g); npar = 4 + n_g;
 *     incoming p1 = (sqrt(s)/2)(1,0,0,1), p2 = (sqrt(s)/2)(1,0,0,-1);
 *   - helicity index h = sum_i bit_i 2^(npar-1-i), bit_i = 1 for physical helicity +1,
 *     particle 0 (g1) is the most significant bit; nhel = 2^npar;
 *   - ME = (1/256) (1/n_g!) sum_{good h} sum_colours |M_h|^2: averaged over the helicities and
 *     colours of the two incoming gluons, divided by n_g! for identical final-state gluons;
 *   - alpha_s fixed (default 0.118), m_t = 173, top width 0 unless set.
 *
 * Momentum layout ("AoSoA", V = 32 events per page): element (event e, particle i, component mu)
 * sits at  mom[((e / 32) * npar + i) * 4 * 32 + mu * 32 + (e % 32)].  A buffer for nevt events
 * holds mg_mom_count(process, nevt) doubles (nevt rounded up to a multiple of 32); pages are
 * 8-byte aligned doubles, every warp-wide access is one 256-byte line.
 *
 * Ownership and errors
 *   - The caller owns every buffer passed in (device buffers are raw cudaMalloc/torch pointers);
 *     the library never frees caller memory.  A context owns only its own state (helicity mask,
 *     colour matrix, couplings, scratch).
 *   - Calls taking a stream are asynchronous and stream-ordered (stream = cudaStream_t, NULL =
 *     legacy default stream).  Argument errors are returned synchronously; launch errors return
 *     MG_ECUDA; device-side conditions (RAMBO non-convergence) are recorded in the context and
 *     reported by mg_check() after the stream has drained.  No C++ exception crosses the ABI.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef MG_H
#define MG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_EINVAL = 1,   /* invalid argument (null pointer, bad size, sqrt(s) <= sum of masses, ...) */
  MG_ENOMEM = 2,   /* device or host allocation failed */
  MG_ECUDA = 3,    /* a CUDA call failed (launch error, no device, ...) */
  MG_ENOCONV = 4,  /* RAMBO massive rescaling did not converge for some event */
  MG_EAGAIN = 5,   /* not ready yet (serving) */
  MG_ETIMEOUT = 6, /* a bounded wait expired */
  MG_EBUSY = 7,    /* resource busy (serving admission) */
  MG_ENOTSUP = 8,  /* valid request that this library does not implement */
  MG_ECANCELED = 9 /* the request was cancelled (serving) */
} mg_status;

typedef enum { MG_GG_TT = 0, MG_GG_TTG = 1, MG_GG_TTGG = 2, MG_GG_TTGGG = 3 } mg_process;

/* Arithmetic of mg_sigmakin.
 *   MG_FP64         plain FP64 throughout (per-event relative error vs an FP64 reference <= 1e-12);
 *   MG_FP32_AMP     amplitudes and colour sum in FP32; FP64 kept for momenta, propagator
 *                   denominators, the top wavefunctions and the helicity sum.  Events whose
 *                   smallest internal invariant (|P^2| of a gluon propagator or |Q^2 - m^2| of a
 *                   quark propagator) is below 3e-4 s -- near-collinear or soft gluons, where FP32
 *                   rounding grows like 1/sqrt(invariant) -- are recomputed (0.1-2 % of the events)
 *                   with double-float (pairs of FP32 values, ~48 bits; MG_LAUNCH_DF_REDO) or FP64
 *                   amplitudes from FP64 per-event data, which keeps every event within 1e-5 of FP64;
 *   MG_FP64_TCCOLOR FP64 amplitudes; colour sum A^dagger C A on the tensor cores: the integer colour
 *                   matrix exact in FP16, every jamp row scaled by a power of two and split hi + lo
 *                   in FP16, FP32 accumulation (~1e-7 relative per helicity);
 *   MG_MIXED        FP32 amplitudes (with the same recomputation) + the tensor-core colour sum.
 * The tensor-core modes need zero top width (MG_ENOTSUP otherwise). */
typedef enum { MG_FP64 = 0, MG_FP32_AMP = 1, MG_FP64_TCCOLOR = 2, MG_MIXED = 3 } mg_precision;

typedef struct {
  double mt;        /* top mass [GeV], default 173 */
  double wt;        /* top width [GeV], default 0 */
  double alphas;    /* strong coupling, default 0.118 */
  int hel_warmup;   /* events used by the helicity filter, default 1024 */
  double hel_tau;   /* helicity h is kept iff max_e |M_h|^2 / sum_h' |M_h'|^2 > hel_tau, default 1e-9 */
} mg_params;

typedef struct mg_ctx mg_ctx;

/* Human-readable name of a status code (static string, never NULL). */
const char* mg_strerror(mg_status s);

/* Fill *p with the defaults listed in mg_params. */
void mg_default_params(mg_params* p);

/* Sizes of a process: npar, nhel, ncol (colour flows = (n_g+2)!), number of Feynman diagrams.
 * Any output pointer may be NULL.  Host only. */
mg_status mg_process_info(mg_process proc, int* npar, int* nhel, int* ncol, int* ndiagrams);

/* Number of doubles of an AoSoA momentum buffer for nevt events (nevt rounded up to 32). */
int64_t mg_mom_count(mg_process proc, int64_t nevt);

/* Exact colour matrix C = num / den (C(sigma,tau) = Tr(T^sigma (T^tau)^dagger), colour flows in
 * the lexicographic order of the gluon permutations; Mangano-Parke colour decomposition).
 * num receives ncol*ncol int64 values, *den the common denominator.  Host only, no GPU needed. */
mg_status mg_colour_matrix(mg_process proc, int64_t* num, int64_t* den);

/* Create a context on the current CUDA device: uploads couplings, colour matrix and helicity
 * tables.  params may be NULL (defaults).  *out receives the context. */
mg_status mg_create(mg_process proc, const mg_params* params, mg_ctx** out);

/* Release a context and its device memory (synchronises the device first).  NULL is a no-op. */
void mg_destroy(mg_ctx* ctx);

/* Philox4x32-10 words (Salmon et al. SC'11) for nevt events and nfinal final-state particles:
 * words[(e * nfinal + j) * 4 + w] = Philox4x32-10(counter {e_lo, e_hi, j, 0}, key {seed_lo, seed_hi})[w].
 * words_dev holds 4 * nevt * nfinal uint32 on the device, 16-byte aligned. */
mg_status mg_philox(uint64_t seed, int64_t nevt, int nfinal, uint32_t* words_dev, void* stream);

/* Random numbers -> momenta (Sec. 1, Fig. 1 of the paper): per event e and final particle j the
 * four uniforms u_w = (x_w + 0.5) 2^-32 of the Philox words above drive massive RAMBO
 * (Kleiss-Stirling-Ellis): massless momenta, then the Newton solve for the rescaling xi,
 * stopped at |f| <= 1e-14 sqrt(s) (<= 50 steps).  Writes AoSoA FP64 momenta of all npar particles
 * (incoming beams included) and, if wgt_dev is not NULL, the phase-space weight per event.
 * sqrt(s) <= 2 m_t -> MG_EINVAL.  Events that fail to converge are counted in the context
 * (see mg_check). */
mg_status mg_rambo(mg_ctx* ctx, uint64_t seed, int64_t nevt, double sqrts, double* mom_dev, double* wgt_dev,
                   void* stream);

/* The same for the events e0 .. e0+nevt-1 of the seed's stream (Philox counters start at e0):
 * event e0+i is written at position i of mom_dev / wgt_dev.  Disjoint ranges on several GPUs
 * reproduce the single-GPU sample exactly. */
mg_status mg_rambo_range(mg_ctx* ctx, uint64_t seed, int64_t e0, int64_t nevt, double sqrts, double* mom_dev,
                         double* wgt_dev, void* stream);

/* Helicity filter (the paper's Sec. 2: the engine sums only the helicities that contribute; which ones do
 * is found once from a sample of events): recompute the context's helicity mask from the first
 * min(nevt, hel_warmup) events of mom_dev (AoSoA).  good(h) <=> max_e |M_h|^2 / sum_h' |M_h'|^2 > hel_tau, the ratios taken in
 * FP64 from FP32-amplitude colour sums (zero top width; FP64 otherwise): with the default hel_tau the kept
 * and the vanishing helicities of these processes are at least six decades apart, so FP32 rounding cannot
 * change the mask.  Stream-ordered; the mask is used by every later mg_sigmakin on this context. */
mg_status mg_hel_filter(mg_ctx* ctx, const double* mom_dev, int64_t nevt, void* stream);

/* Matrix elements (the per-event hot path of the paper's Sec. 2, its "sigmaKin": every tree diagram,
 * colour sum and helicity sum of one event; throughput N_events / t_MEs, Tables 1-2): me_dev[e] = ME of
 * event e of mom_dev (AoSoA), e < nevt.  If no helicity mask has been computed yet, the first call runs
 * mg_hel_filter on its own first events.  precision selects the arithmetic (MG_ENOTSUP if not built). */
mg_status mg_sigmakin(mg_ctx* ctx, const double* mom_dev, int64_t nevt, mg_precision precision, double* me_dev,
                      void* stream);

/* The same, through host buffers: copies mom_host (AoSoA, mg_mom_count doubles) to the device,
 * computes, and copies the MEs back to me_host; returns after the results are in me_host.
 * Batches of 32,768 events or more are split into up to 4 chunks of whole 32-event pages (each of at
 * least 16,384 events): the momenta of later chunks are copied in and the MEs of earlier ones copied
 * out (on two copy streams of the context) while a chunk's MEs are computed on `stream`.  The results
 * are those of one mg_sigmakin call over the batch.  Pinned host buffers are needed for the copies to
 * overlap.  Device staging buffers are owned by the context and grown on demand. */
mg_status mg_sigmakin_host(mg_ctx* ctx, const double* mom_host, int64_t nevt, mg_precision precision,
                           double* me_host, void* stream);

/* The helicity mask of the filter above (paper Sec. 2; a test and diagnostics hook): copy the current mask
 * (ceil(nhel/32) words, bit h of word h/32) to mask_host and the number of good helicities to *ngood.
 * Synchronises the context's last stream. */
mg_status mg_hel_mask(mg_ctx* ctx, uint32_t* mask_host, int* ngood);

/* Device-side conditions of the random numbers -> momenta -> ME workflow (paper Sec. 1, Fig. 1) that a
 * stream-ordered call cannot return synchronously.
 * Wait for the context's work on stream and report device-side conditions: MG_ETIMEOUT if a bounded
 * wait inside the tensor-memory colour kernel gave up (its results are then invalid), MG_ENOCONV if any
 * event since the last mg_check failed to converge in RAMBO (the count goes to *nbad if not
 * NULL), MG_ECUDA on an asynchronous CUDA error, else MG_OK.  Clears the conditions. */
mg_status mg_check(mg_ctx* ctx, void* stream, int64_t* nbad);

/* Floating-point operations of one event's matrix element in this engine's algorithm for the given
 * precision (the roofline numerator): *amp_flops for the per-event wavefunctions and propagators
 * (once per event) and the currents and jamps of every gluon-helicity combination with a good
 * helicity, *colour_flops for the colour sums (4 ncol(ncol+1)/2 + 4 ncol per good helicity), counting
 * an FMA as 2.  The FP64-amplitude modes tabulate (gamma.J) v per current, the FP32-amplitude modes
 * form it per jamp term; from gg -> t tbar g on, the FP64-amplitude count is that of the
 * default MG_LAUNCH_SHARED algorithm (the currents of fewer than all gluons, with their (gamma.J) v, once
 * per helicity assignment of their own gluons per event).  mask (ceil(nhel/32) words, as returned by
 * mg_hel_mask) selects the good helicities; NULL = all.  Host only. */
mg_status mg_flops_per_event(mg_process proc, mg_precision precision, const uint32_t* mask, double* amp_flops,
                             double* colour_flops);

/* As mg_flops_per_event, for the algorithm that the launch flags `flags` (MG_LAUNCH_* bits, as
 * mg_get_launch_shape returns them) select: with MG_LAUNCH_SHARED the FP64-amplitude modes count the
 * shared currents once per helicity assignment of their own gluons, without it once per good
 * gluon-helicity combination.  flags < 0 = the defaults of mg_create.  Host only. */
mg_status mg_flops_per_event_shape(mg_process proc, mg_precision precision, const uint32_t* mask, int flags,
                                   double* amp_flops, double* colour_flops);

/* FP64 matrix elements exactly as mg_sigmakin(..., MG_FP64, ...), for callers that must not have
 * the library allocate device memory during the call (an application that hands the engine a
 * fixed memory budget, or whose own pooling allocator must remain the only one): this entry point
 * calls no cudaMalloc/cudaFree and no allocating routine.  The paper has no counterpart; it is an
 * integration aid of this library.
 *   - Scratch: a fixed 16 MiB array in device global memory (2^21 doubles), part of the library
 *     image, so every GPU that loads the library holds it until the process exits.  A call needs
 *     nhel * ceil(nevt/32)*32 <= 2^21, i.e. nevt <= 131072 (gg->tt), 65536 (gg->ttg),
 *     32768 (gg->ttgg), 16384 (gg->ttggg); larger batches return MG_EINVAL: split them.
 *   - The context must already hold a helicity mask (mg_hel_filter, or one earlier mg_sigmakin),
 *     else MG_EINVAL.
 *   - All calls on a device share the one scratch array (it keeps the last call's contents; every
 *     element a call reads is written by that call first).  Calls whose work can overlap on the
 *     GPU (different streams without ordering, several host threads) race on it: serialise them.
 *   - The first call on each device looks up the array's device address (cudaGetSymbolAddress with
 *     that device current); make that first call before any stream capture.
 *   - The library allocates nothing, but the CUDA driver itself may enlarge the context's
 *     per-thread local-memory reservation the first time a kernel with a large stack runs in the
 *     process (the five-gluon kernel keeps ~28 KB of local arrays per thread), which is a device
 *     allocation and a device-wide synchronisation made by the driver.  To keep that out of the
 *     caller's steady state, make one warm-up call per device and process at set-up. */
mg_status mg_sigmakin_noalloc(mg_ctx* ctx, const double* mom_dev, int64_t nevt, double* me_dev, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Event-level epilogues (the paper's Sec. 4: event-by-event helicities and leading colours are the two
 * pieces its GPU matrix elements still lacked for unweighted-event (LHE) files; Sec. 2: the running of
 * the QCD coupling alpha_s is a feature the engine gained).  FP64 matrix elements.
 * --------------------------------------------------------------------------------------------- */

/* FP64 matrix elements (as mg_sigmakin(..., MG_FP64, ...), summed over the good helicities in ascending
 * helicity index) with, per event e:
 *   - hel_dev[e] (if not NULL): the helicity chosen with probability |M_h|^2 / sum_h' |M_h'|^2 -- the
 *     smallest good h whose running sum over good helicities (ascending h) of the colour-summed |M_h|^2
 *     exceeds rnd_hel_dev[e] times the total; index convention of this header;
 *   - col_dev[e] (if not NULL): the leading-colour flow chosen with probability w_sigma / sum w, where
 *     w_sigma = sum over good helicities of |J_sigma(h)|^2 (the colour-ordered amplitude of flow sigma,
 *     the lexicographic rank of the gluon ordering along the quark line, see mg_colour_flow) -- the
 *     smallest sigma whose running sum of w exceeds rnd_col_dev[e] times the total;
 *   - running_alphas = 1: the matrix element at the one-loop running coupling alpha_s(mu_e), mu_e = H_T/2
 *     (half the sum over t, tbar and the final-state gluons of sqrt(m^2 + px^2 + py^2)),
 *     alpha_s(mu) = a / (1 + a b0 ln(mu^2 / M_Z^2)), a = params.alphas taken as alpha_s(M_Z),
 *     M_Z = 91.1876 GeV, b0 = (33 - 2 n_f)/(12 pi), n_f = 5 -- i.e. the fixed-coupling matrix element
 *     times (alpha_s(mu_e)/a)^(n_g+2), every tree diagram carrying g_s^(n_g+2); running_alphas = 0: the
 *     fixed coupling params.alphas.  alphas_dev[e] (if not NULL) receives the coupling used.
 * rnd_hel_dev / rnd_col_dev: caller-supplied uniform numbers in [0, 1), one per event (device, FP64;
 * needed when the matching output is requested, else MG_EINVAL).  hel_dev / col_dev: int32 per event.
 * Every buffer holds nevt entries.  Zero top width only (MG_ENOTSUP otherwise).  The matrix elements come
 * from the FP64 algorithm that the context's MG_FP64 launch shape selects (with MG_LAUNCH_SHARED: the
 * shared currents and quark-line prefixes); at fixed coupling they equal mg_sigmakin(MG_FP64)'s up to the
 * order of the helicity sum.
 * Scratch: per-slot sums of |J_sigma|^2 (events processed in chunks that keep it within 1 GiB, and the
 * shared currents within 2 GiB), owned by the context.  If no helicity mask exists yet, the call first
 * runs mg_hel_filter on its own first events. */
mg_status mg_sigmakin_lhe(mg_ctx* ctx, const double* mom_dev, int64_t nevt, const double* rnd_hel_dev,
                          const double* rnd_col_dev, int running_alphas, double* me_dev, int* hel_dev, int* col_dev,
                          double* alphas_dev, void* stream);

/* Running coupling for matrix elements of any precision mode, in place: me_dev[e] *= (alpha_s(mu_e)/a)^(n_g+2)
 * with mu_e, alpha_s(mu) and a as in mg_sigmakin_lhe; alphas_dev (may be NULL) receives alpha_s(mu_e).
 * mom_dev: the events' AoSoA momenta. */
mg_status mg_alphas_running(mg_ctx* ctx, const double* mom_dev, int64_t nevt, double* me_dev, double* alphas_dev,
                            void* stream);

/* Single-diagram-enhancement channel weights (MadEvent's phase-space channels; the paper's Sec. 2 lists the
 * algorithm among the engine's features).  Channel d is a Feynman diagram built from three-point vertices
 * only (3 / 15 / 105 / 945 for n_g = 0..3; a diagram with a four-gluon vertex has no propagator structure of
 * its own and is no channel): an ordered list of binary gluon trees attached along the quark line from the
 * top to the antitop, the trees' gluons partitioning the gluons.  Per event e (FP64):
 *     w_dev[d * nevt + e] = sum_h |A_d(h)|^2 / sum_d' sum_h |A_d'(h)|^2   (good helicities h),
 * A_d the diagram's amplitude with its colour factor stripped (Feynman-gauge vertices and propagators; the
 * couplings and phases, common to all channels, cancel).  w_dev holds nchannels * nevt doubles.  Zero top
 * width (MG_ENOTSUP otherwise); if no helicity mask exists yet, the call first runs mg_hel_filter on its
 * own first events.  Scratch (events in chunks of at most 2 GiB of per-channel sums) is owned by the context. */
mg_status mg_sde_weights(mg_ctx* ctx, const double* mom_dev, int64_t nevt, double* w_dev, void* stream);

/* Number of channels of a process.  Host only. */
mg_status mg_sde_channels(mg_process proc, int* nchannels);

/* The channel's diagram as text into key (keylen bytes, NUL-terminated; MG_EINVAL if too short): its gluon
 * trees in quark-line order from the top, joined by "|"; a tree is a gluon label (1, 2 the incoming gluons,
 * 3.. the final-state ones) or "(A,B)", the child holding the smaller label first.  E.g. for gg -> t tbar:
 * "1|2", "2|1", "(1,2)".  Host only. */
mg_status mg_sde_channel_key(mg_process proc, int channel, char* key, int keylen);

/* The gluon ordering of colour flow `flow` (0 <= flow < (n_g+2)!): order[i] = gluon label (0 = g1, 1 = g2,
 * 2.. = final-state gluons g3..) at position i along the quark line, flow = lexicographic rank of the
 * permutation; the flow's colour factor is (T^{a_order[0]} ... T^{a_order[K-1]})_{i_t j_tbar}.  Host only. */
mg_status mg_colour_flow(mg_process proc, int flow, int* order);

/* ---------------------------------------------------------------------------------------------
 * Launch-shape autotuner and CUDA-graph batches (no counterpart in the paper; its Sec. 4 and
 * Fig. 2 show the throughput depending on how many events one launch holds).
 * --------------------------------------------------------------------------------------------- */

/* Launch options of the matrix-element kernel (the flags of mg_get/set_launch_shape):
 *   MG_LAUNCH_UNROLLED  the kernel with the recursion unrolled at compile time, where built (FP32
 *                       amplitudes of gg -> t tbar, t tbar g and t tbar g g; elsewhere the flag falls
 *                       back to the kernel that reads the recursion tables at run time);
 *   MG_LAUNCH_DF_REDO   FP32 modes: the events recomputed for a small internal invariant get
 *                       double-float amplitudes (FP32 pipe) instead of FP64 ones (FP64 pipe, which
 *                       otherwise idles beside the FP32 launch);
 *   MG_LAUNCH_FUSED     with MG_LAUNCH_UNROLLED: the per-event FP64 record is computed inside the
 *                       matrix-element kernel (32 events per block; tile_ev and slot_major unused), so
 *                       that its FP64 work overlaps the FP32 work of other blocks;
 *   MG_LAUNCH_WARP      FP32 amplitudes of gg -> t tbar + 1..3 gluons: one group of lanes (4, 8 or 32 for
 *                       1, 2 or 3 final-state gluons) per (event, gluon-helicity combination), its
 *                       currents and jamps in shared memory, the work split over the lanes (takes
 *                       precedence over MG_LAUNCH_UNROLLED); with MG_MIXED it also sums the colours on
 *                       the tensor cores itself, unless
 *   MG_LAUNCH_TC_APART  MG_MIXED with MG_LAUNCH_WARP: write the jamps out for the separate tensor-core
 *                       colour kernel instead;
 *   MG_LAUNCH_SHARED    MG_FP64: the gluon currents of fewer than all gluons (and their products with the
 *                       antitop spinors) are computed once per helicity assignment of their own gluons, by
 *                       a pass before the matrix-element kernel, instead of once per gluon-helicity
 *                       combination;
 *   MG_LAUNCH_TC_SYNC   the separate tensor-core colour pass (MG_FP64_TCCOLOR, and MG_MIXED where the jamps
 *                       are written out) on warp-level mma.sync instead of the default fifth-generation
 *                       tensor-core kernel (tcgen05.mma with the accumulators in tensor memory). */
#define MG_LAUNCH_UNROLLED 1
#define MG_LAUNCH_DF_REDO 2
#define MG_LAUNCH_FUSED 4
#define MG_LAUNCH_WARP 8
#define MG_LAUNCH_TC_APART 16
#define MG_LAUNCH_SHARED 32
#define MG_LAUNCH_TC_SYNC 64

/* Time mg_sigmakin(precision) of nevt probe events (this context's process, fixed seed) for each
 * launch shape of the matrix-element kernel -- 32, 64 or 128 events per 128-thread block (the other
 * threads of a block take further helicity combinations of the same events), grid dispatched
 * event-tile-major or helicity-tile-major, with and without MG_LAUNCH_UNROLLED where that kernel
 * exists, MG_LAUNCH_UNROLLED | MG_LAUNCH_FUSED, MG_LAUNCH_WARP and (MG_MIXED) MG_LAUNCH_WARP | MG_LAUNCH_TC_APART
 * -- then the fastest with MG_LAUNCH_DF_REDO (FP32 modes) or MG_LAUNCH_SHARED (MG_FP64) toggled, and for the
 * tensor-core colour modes with MG_LAUNCH_TC_SYNC toggled, and keep the fastest
 * for this context and precision.  cache_path (may be NULL): text file of
 * "gpu|process|precision tile_ev slot_major flags ms" lines; an existing entry is used without timing,
 * a new result is appended.  *best_ms may be NULL.  Synchronous; allocates probe buffers; nevt >= 32. */
mg_status mg_autotune(mg_ctx* ctx, mg_precision precision, int64_t nevt, const char* cache_path, double* best_ms);

/* The launch shape mg_sigmakin(precision) uses on this context (default: 128 events per block,
 * event-tile-major, flags MG_LAUNCH_UNROLLED | MG_LAUNCH_DF_REDO | MG_LAUNCH_FUSED, plus MG_LAUNCH_SHARED
 * for gg -> t tbar g, t tbar g g and t tbar g g g, MG_LAUNCH_WARP for t tbar g g and t tbar g g g, and
 * MG_LAUNCH_TC_APART for t tbar g g g).  Any out-pointer may be NULL. */
mg_status mg_get_launch_shape(mg_ctx* ctx, mg_precision precision, int* tile_ev, int* slot_major, int* flags);

/* Set the launch shape of mg_sigmakin(precision) by hand: tile_ev in {32, 64, 128}, slot_major 0 or 1,
 * flags a combination of the MG_LAUNCH_ bits.  MG_EINVAL otherwise. */
mg_status mg_set_launch_shape(mg_ctx* ctx, mg_precision precision, int tile_ev, int slot_major, int flags);

/* FP32 modes (MG_FP32_AMP, MG_MIXED): the events whose smallest internal invariant -- |P^2| of a gluon
 * propagator or |Q^2 - m_t^2| of a top propagator, evaluated from the momenta -- is below tau * s are
 * recomputed with double-float (or FP64) amplitudes; default 3e-4, and 3e-5 for gg -> t tbar g g g, where
 * the plain FP32 error of the events kept was measured <= 4e-6; tau = 0 recomputes nothing (the plain
 * FP32 error).  MG_EINVAL for tau < 0 or not finite. */
mg_status mg_set_fp32_tau(mg_ctx* ctx, double tau);

/* One job of a graph batch: the step mg_rambo_range(seed, e0, nevt, sqrts, mom_dev) ->
 * mg_hel_filter(mom_dev, nevt) -> mg_sigmakin(precision, me_dev) on ctx.  Every job of a batch needs
 * its own context. */
typedef struct {
  mg_ctx* ctx;
  uint64_t seed;
  int64_t e0, nevt;
  double sqrts;
  double* mom_dev;
  double* me_dev;
  mg_precision precision;
} mg_job;

typedef struct mg_graph mg_graph;

/* One job of mg_sigmakin_batch: the FP64 matrix elements of nevt events (AoSoA momenta) on ctx. */
typedef struct {
  mg_ctx* ctx;
  const double* mom_dev;
  int64_t nevt;
  double* me_dev;
} mg_batch_job;

/* FP64 matrix elements of njobs jobs (1..64, any mix of processes, one context each, zero top width) with
 * ONE persistent kernel launch for all their matrix elements: its thread blocks drain a queue of (job,
 * gluon-helicity slot, 128-event tile) work items (the jobs with more gluons first) from an atomic counter,
 * so many small jobs fill the GPU together (the paper's Sec. 4: throughput keeps growing up to batches of
 * ~16k events).  Per job, as mg_sigmakin(MG_FP64): the helicity filter on its own first events if its
 * context has no mask yet, the per-event records, and the helicity sums after the shared launch.  Results
 * are bit-identical to mg_sigmakin(MG_FP64) with a launch shape without MG_LAUNCH_SHARED.  Stream-ordered,
 * graph-capturable once each context's scratch is large enough (mg_graph_create reserves it). */
mg_status mg_sigmakin_batch(const mg_batch_job* jobs, int njobs, void* stream);

/* Flags of mg_graph_create_ex. */
#define MG_GRAPH_PERSISTENT 1   /* FP64 jobs: every job's matrix elements in one mg_sigmakin_batch launch */

/* Capture the steps of njobs jobs (any mix of processes) into ONE CUDA graph, each job on its own
 * parallel branch; all scratch is reserved first, so launching the graph allocates nothing. */
mg_status mg_graph_create(const mg_job* jobs, int njobs, mg_graph** out);

/* As mg_graph_create; flags = MG_GRAPH_PERSISTENT (every job MG_FP64 with zero top width, at most 64 jobs,
 * else MG_ENOTSUP / MG_EINVAL): each job's mg_rambo_range and mg_hel_filter on its own branch, then the
 * matrix elements of all jobs in one persistent launch (mg_sigmakin_batch) and the helicity sums.
 * mg_graph_update, _launch, _nodes and _destroy apply unchanged. */
mg_status mg_graph_create_ex(const mg_job* jobs, int njobs, int flags, mg_graph** out);

/* Replace the jobs' parameters (seeds, event ranges, sizes of an identical topology) in place
 * (cudaGraphExecUpdate); MG_EINVAL if the new jobs do not fit the captured topology. */
mg_status mg_graph_update(mg_graph* g, const mg_job* jobs, int njobs);

/* One cudaGraphLaunch of the whole batch on stream; asynchronous. */
mg_status mg_graph_launch(mg_graph* g, void* stream);

/* Number of nodes (kernels, memsets, event waits) in the captured graph. */
mg_status mg_graph_nodes(mg_graph* g, int* nodes);

void mg_graph_destroy(mg_graph* g);

/* ---------------------------------------------------------------------------------------------
 * Serving: continuous batching of matrix-element requests (no counterpart in the paper, which runs
 * one batch at a time; the paper's Sec. 4 notes that 8k-event batches underfill a GPU).
 * A request (process, seed, nevt) returns the MEs of events 0..nevt-1 of the seed's Philox stream
 * (mg_rambo_range + mg_sigmakin) with the server's resident helicity mask of the process: computed once,
 * when the server is created, by mg_hel_filter on the first params.hel_warmup events of Philox seed
 * MG_SERVE_MASK_SEED (at cfg.sqrts), and shared by every slot.  A scheduler
 * thread admits queued requests in FIFO order when a slot is free and the sum of the in-flight
 * requests' device footprints (mg_serve_footprint) stays within hbm_cap_bytes; each slot is a CUDA
 * stream with its own pre-reserved contexts and buffers, so admitted requests run concurrently on
 * the GPU and serving itself allocates no device memory.  A request's result does not depend on
 * what else is in flight.  The server is thread-safe; results are returned through host memory.
 * --------------------------------------------------------------------------------------------- */
typedef struct {
  int slots;               /* requests in flight at once (CUDA streams), 1..64, default 8 */
  int64_t max_nevt;        /* events per launch; larger requests run in consecutive chunks; default 65536 */
  int64_t hbm_cap_bytes;   /* admission cap on the in-flight device footprint, default 64 GiB */
  mg_precision precision;  /* arithmetic of every request, default MG_FP64 */
  double sqrts;            /* collision energy [GeV], default 1500 */
  mg_params params;        /* physics parameters, default mg_default_params */
} mg_serve_cfg;

typedef struct mg_server mg_server;

/* Philox seed of the warm-up events from which a server computes its helicity masks. */
#define MG_SERVE_MASK_SEED 0x4D47u

void mg_serve_default_cfg(mg_serve_cfg* cfg);

/* Device bytes a request of nevt events holds while in flight (momenta, MEs, scratch); host only. */
int64_t mg_serve_footprint(mg_process proc, int64_t nevt, mg_precision precision);

/* Create a server on the current device (allocates every slot up front).  cfg may be NULL. */
mg_status mg_serve_create(const mg_serve_cfg* cfg, mg_server** out);

/* Queue a request; *ticket identifies it.  Returns at once. */
mg_status mg_serve_submit(mg_server* srv, mg_process proc, uint64_t seed, int64_t nevt, uint64_t* ticket);

/* Non-blocking: *done = 0 while in flight; once done, *done = 1, the nevt MEs are copied to
 * me_out_host (if not NULL), *latency_ms (if not NULL) receives completion - submission time, the
 * request is released and its status returned (MG_ENOCONV if RAMBO failed for some event). */
mg_status mg_serve_poll(mg_server* srv, uint64_t ticket, double* me_out_host, int* done, double* latency_ms);

/* Blocking version with a timeout: MG_ETIMEOUT (request kept) if not done within timeout_ms. */
mg_status mg_serve_wait(mg_server* srv, uint64_t ticket, double* me_out_host, int64_t timeout_ms, double* latency_ms);

/* Cancel a request.  A queued request is dropped before it starts; one in flight stops at the next chunk
 * boundary (the chunk on the device runs to its end: nothing is interrupted).  Its poll or wait then
 * returns MG_ECANCELED with the MEs of the chunks that finished and zeros for the rest (a request whose
 * last chunk was already running completes normally).  MG_OK if the request was cancelled or had already
 * finished, MG_EINVAL for an unknown ticket.  Returns at once. */
mg_status mg_serve_cancel(mg_server* srv, uint64_t ticket);

/* Counters since creation: completed requests (cancelled ones included), the events computed for them,
 * peak in-flight footprint and count. */
mg_status mg_serve_stats(mg_server* srv, int64_t* completed, int64_t* events, int64_t* peak_bytes, int* peak_inflight);

/* Drain the queue, stop the scheduler and free everything (unpolled results are dropped). */
void mg_serve_destroy(mg_server* srv);

/* Diagnostic: FMA throughput of the current device, the ALU roofline denominator of the
 * matrix-element kernels.  Runs 8 independent FMA chains per thread (iters x 16 FMAs each) over
 * 8 blocks of 256 threads per SM and returns the measured rate in flop/s (an FMA counts 2) for
 * FP64 (fp32 = 0) or FP32 (fp32 = 1).  Synchronous; 1 <= iters <= 2^20. */
mg_status mg_measure_fma_peak(int fp32, int iters, double* flops_per_s);

/* Diagnostic: dense FP16 tensor-core throughput of the current device through the instruction the colour
 * pass uses (tcgen05.mma kind::f16, FP32 accumulators in tensor memory): one CTA per SM issues iters MMAs
 * of M = 128, N = 256, K = 16 into one accumulator; returns the rate in flop/s (2 M N K per MMA).  The
 * operands are small integers, so the accumulated result is exact and is checked on the host: MG_ECUDA
 * if it differs, MG_ETIMEOUT if a bounded wait ran out.  Synchronous; 1 <= iters <= 65536. */
mg_status mg_measure_mma_peak(int iters, double* flops_per_s);

/* Diagnostic: the number of CUDA kernels this library has launched in this process, on every
 * context, stream and thread (a launch captured into a CUDA graph counts once, at capture; graph
 * replays do not count).  The difference of two reads brackets the launches of the calls between
 * them.  Host only; never fails. */
int64_t mg_kernel_launches(void);

/* Diagnostics of the failure paths (no counterpart in the paper).
 *
 * Host-side allocation-failure injector: the nth device or pinned-host allocation that the library makes
 * from now on (nth = 1: the next one) fails as an exhausted device would, and the call that made it
 * returns MG_ENOMEM after freeing what it had allocated; later allocations succeed again.  nth = 0
 * disarms it.  Process-wide; MG_EINVAL for nth < 0.  No GPU needed. */
mg_status mg_diag_fail_alloc(int64_t nth);

/* Device and pinned-host allocations of the library alive now (process-wide): every context, server and
 * graph returns to the count it found when destroyed, including after a failed creation. */
int64_t mg_diag_live_allocs(void);

/* With on = 1 the tensor-memory colour
 * pass on this context issues no MMAs, so each CTA's bounded mbarrier wait runs out (after 0.2 s): the
 * kernel records it, frees its tensor memory and returns; mg_check then reports MG_ETIMEOUT and the
 * context stays usable.  on = 0 restores normal operation.  Host only; no fault, trap or hang. */
mg_status mg_diag_tc_stall(mg_ctx* ctx, int on);

#ifdef __cplusplus
}
#endif

#endif /* MG_H */
