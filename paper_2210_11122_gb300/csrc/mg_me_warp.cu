// mg_me_warp.cu -- FP32 matrix-element kernel with one lane group (a warp or part of one) per (event,
// gluon-helicity slot).
//
// Same physics, record input and outputs as the per-thread kernels (mg_me_kernel.cuh, mg_me3.cu), for
// processes whose per-slot state does not fit in a thread: with 5 gluons a slot carries 105 gluon
// currents, 60 all-gluon currents and 4 x 120 jamps (~9 KB), which a thread can only keep in local
// memory (spilled to L2 and DRAM at the occupancy the FP32 pipe needs).  Here the G lanes of a group
// (G = 32 for 5 gluons, 8 for 4, 4 for 3) share that state in shared memory and split the work:
//   * currents level by level (all sequences of one length are independent): one sequence per lane;
//   * the quark-line walk: the first half of the group takes top helicity -, the second half top
//     helicity +, each lane a contiguous run of colour orderings (prefix spinors shared along the run,
//     in registers);
//   * the colour sums of the four helicities together: rows of C A per lane (register-blocked over
//     rows and helicities), then sums over the group; or (jamp output) the jamps are written out for
//     the tensor-core colour sum.
#include <atomic>
#include <type_traits>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "mg_internal.h"
#include "mg_kernels.h"
#include "mg_me_algebra.cuh"

namespace mg {
namespace wk {

// Two FP32 values in one 64-bit register pair, and the paired fused multiply-add d = a b + c of each half
// (Blackwell's FFMA2: one instruction for two FP32 FMAs)
__device__ __forceinline__ uint64_t pack2(float2 v) {
  return (static_cast<uint64_t>(__float_as_uint(v.y)) << 32) | __float_as_uint(v.x);
}
__device__ __forceinline__ float2 unpack2(uint64_t v) {
  return make_float2(__uint_as_float(static_cast<uint32_t>(v)), __uint_as_float(static_cast<uint32_t>(v >> 32)));
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}


using v2::cx;

constexpr int kWarps = 4;   // warps per block; a block holds slots of one event

// lanes per slot G: the work of one slot spread over as many lanes as its widest stage keeps busy
template <int K> struct WSizes;
template <> struct WSizes<3> { static constexpr int ncol = 6, nseq = 6, nfull = 3, G = 4; };
template <> struct WSizes<4> { static constexpr int ncol = 24, nseq = 22, nfull = 12, G = 8; };
template <> struct WSizes<5> { static constexpr int ncol = 120, nseq = 105, nfull = 60, G = 32; };

// Shared-memory storage of a complex current component: float2 for FP32 amplitudes, float4 (hi and lo
// of the real, then of the imaginary part) for double-float ones (the recomputation of flagged events)
template <class T> struct WStore;
template <> struct WStore<float> { using type = float2; };
template <> struct WStore<dd::df> { using type = float4; };
__device__ __forceinline__ cx<float> ldw(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ cx<dd::df> ldw(float4 v) { return {dd::df(v.x, v.y), dd::df(v.z, v.w)}; }
__device__ __forceinline__ float2 stw(cx<float> v) { return make_float2(v.r, v.i); }
__device__ __forceinline__ float4 stw(cx<dd::df> v) { return make_float4(v.r.hi, v.r.lo, v.i.hi, v.i.lo); }
// a jamp rounded to FP32 for the colour sum (FP32 arithmetic either way: C is exact, the quadratic form
// is well conditioned)
__device__ __forceinline__ float2 jamp32(cx<float> v) { return make_float2(v.r, v.i); }
__device__ __forceinline__ float2 jamp32(cx<dd::df> v) {
  return make_float2(__fadd_rn(v.r.hi, v.r.lo), __fadd_rn(v.i.hi, v.i.lo));
}
// the per-event record: FP32 values for FP32 amplitudes, FP64 for double-float ones
template <class T> struct WRec { using type = float; };
template <> struct WRec<dd::df> { using type = double; };
__device__ __forceinline__ float rec_val(float v, float*) { return v; }
__device__ __forceinline__ dd::df rec_val(double v, dd::df*) { return dd::df(v); }

// The recursion tables (18 KB) are copied into shared memory for 5 gluons and read through L1 otherwise:
// with 4 gluons the copy costs a resident block per SM (measured 3 % slower), with 5 the table reads
// of the 32-lane groups are faster from shared memory (measured 3 % faster)
template <int K> constexpr bool kTabSmem = K == 5;

// shared state of one slot: component-major, so that lanes reading different currents hit different banks
template <int K, class T = float>
struct SlotState {
  using W = typename WStore<T>::type;
  W J[4][WSizes<K>::nseq];
  W JF[4][WSizes<K>::nfull];
  float2 A[4][WSizes<K>::ncol];   // jamps of helicity 2 * top + antitop (FP32)
};

__device__ __forceinline__ cx<float> c2(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 f2(cx<float> v) { return make_float2(v.r, v.i); }


// first canonical sequence of length L (sequences are numbered by length: K singles, then L = 2, 3, ...)
__host__ __device__ constexpr int seq_start(int K, int L) {
  int s = K;
  for (int l = 2; l < L; ++l) {
    int n = 1;
    for (int i = 0; i < l; ++i) n *= K - i;
    s += n / 2;
  }
  return L <= 1 ? 0 : s;
}

// Epilogues: the colour sums in FP32 on the FP32 pipe (SIMT), the jamps written out for the separate
// tensor-core colour kernel (JAMPS), or the colour sums on the tensor cores inside this kernel (MMA)
enum Epi { kSimt = 0, kJamps = 1, kMma = 2 };

// 2^k as a double, built from its exponent bits (exact; |k| < 1000): undoes a power-of-two row scale
// with one multiplication instead of an FP64 division
__device__ __forceinline__ double pow2d(int k) { return __longlong_as_double(static_cast<long long>(1023 + k) << 52); }

// 2^k as a float from its exponent bits (exact), 0 below the normal range; k <= 0 here
__device__ __forceinline__ float pow2f_neg(int k) {
  return k >= -126 ? __uint_as_float(static_cast<unsigned>(127 + k) << 23) : 0.f;
}

// s 2^E as a double, built from the IEEE 754 fields of the float s (exact: the mantissa is copied and
// the exponent moved), without an FP64 instruction for normal s; zero and FP32 subnormals take the
// FP64 route
__device__ __forceinline__ double f32_times_pow2(float s, int E) {
  const unsigned u = __float_as_uint(s);
  const unsigned ef = (u >> 23) & 0xffu;
  if ((u & 0x7fffffffu) == 0) return 0.0;   // E may be a placeholder here
  if (ef == 0) return static_cast<double>(s) * pow2d(E);
  const unsigned long long bits = (static_cast<unsigned long long>(u >> 31) << 63) |
                                  (static_cast<unsigned long long>(static_cast<int>(ef) - 127 + E + 1023) << 52) |
                                  (static_cast<unsigned long long>(u & 0x7fffffu) << 29);
  return __longlong_as_double(static_cast<long long>(bits));
}

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ uint32_t pack_h2(__half lo_half, __half hi_half) {
  return static_cast<uint32_t>(__half_as_ushort(lo_half)) | (static_cast<uint32_t>(__half_as_ushort(hi_half)) << 16);
}
__device__ __forceinline__ float unsplit(uint32_t h, uint32_t l, int k) {
  const __half hh = __ushort_as_half(static_cast<unsigned short>(k ? h >> 16 : h & 0xffffu));
  const __half lh = __ushort_as_half(static_cast<unsigned short>(k ? l >> 16 : l & 0xffffu));
  return fmaf(__half2float(lh), 1.f / 2048.f, __half2float(hh));
}

template <int K, class T = float>
struct SmemLayout {
  static constexpr int GPW = 32 / WSizes<K>::G;
  static constexpr size_t rec_off = sizeof(SlotState<K, T>) * kWarps * GPW;
  static constexpr size_t tab_off =
      (rec_off + sizeof(typename WRec<T>::type) * v2::EvLayout<K>::NBASE + 15) / 16 * 16;
  static constexpr size_t bytes = kTabSmem<K> ? tab_off + sizeof(Tables) : tab_off;
};

// 4 resident blocks per SM for FP32 amplitudes: each block's shared memory plus the 1 KB the hardware
// reserves per block within the SM's 228 KB
static_assert(SmemLayout<4>::bytes + 1024 <= 233472 / 4 && SmemLayout<5>::bytes + 1024 <= 233472 / 4,
              "FP32 lane-group kernel: shared memory for 4 blocks per SM");

// T = float: the FP32-amplitude kernel, one block per event (blockIdx.x), record from k_event_prep.
// T = dd::df: the recomputation of the flagged events (evlist[0 .. *nlist)) with double-float amplitudes:
// each block walks the list with a stride of gridDim.x, computes the event's FP64 record in shared memory
// (four threads, one record part each) and runs the same slot work; SIMT colour epilogue only.
// (resident blocks per SM: 4 for FP32 (the shared memory allows that many) and the registers to match;
// 2 for double-float, whose state is twice as large)
template <int K, int EPI, class T = float>
__global__ void __launch_bounds__(kWarps * 32, std::is_same<T, float>::value ? 4 : 2)
k_me_warp(const void* __restrict__ rec_any, int64_t nevt, const Tables* __restrict__ tab_g, const int* __restrict__ gslots,
          const int* __restrict__ nslot_dev, const uint32_t* __restrict__ mask, const float* __restrict__ cfull,
          const __half* __restrict__ cmat16, MeConst cst, double* __restrict__ out, int64_t stride,
          float2* __restrict__ jout, const uint8_t* __restrict__ skip, const int* __restrict__ evlist = nullptr,
          const int* __restrict__ nlist = nullptr, int rows_out = 0) {
  constexpr bool DF = std::is_same<T, dd::df>::value;
  static_assert(!DF || EPI == kSimt, "double-float: SIMT colour sums only");
  using RecT = typename WRec<T>::type;
  using L = v2::EvLayout<K>;
  constexpr int npar = K + 2, NCOL = WSizes<K>::ncol, NFULL = WSizes<K>::nfull;
  constexpr int NSUB = 1 << K;
  constexpr int G = WSizes<K>::G, GPW = 32 / G;   // lanes per slot, slots per warp
  // shared memory (dynamic, SmemLayout): the slots' state, the event's record (read by every slot of the
  // block) and, for 5 gluons, the recursion tables (read with per-lane indices)
  extern __shared__ __align__(16) unsigned char wsm[];
  SlotState<K, T>* sh = reinterpret_cast<SlotState<K, T>*>(wsm);
  RecT* rs = reinterpret_cast<RecT*>(wsm + SmemLayout<K, T>::rec_off);
  Tables& tabs = *reinterpret_cast<Tables*>(wsm + SmemLayout<K, T>::tab_off);
  const int warp = threadIdx.x >> 5, grp = (threadIdx.x & 31) / G, lane = threadIdx.x % G;
  const unsigned gmask = (G == 32 ? 0xffffffffu : ((1u << (G & 31)) - 1u)) << (grp * G);   // this group's lanes
  const int slot0 = (blockIdx.y * kWarps + warp) * GPW;   // the warp's first slot
  const int slot = slot0 + grp;
  const int nslot = *nslot_dev;
  if constexpr (DF) {
    if (static_cast<int>(blockIdx.x) >= *nlist) return;   // no listed event for this block
  }
  if constexpr (kTabSmem<K>) {
    static_assert(sizeof(Tables) % 4 == 0, "table copy in words");
    const unsigned* src = reinterpret_cast<const unsigned*>(tab_g);
    unsigned* dst = reinterpret_cast<unsigned*>(&tabs);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(Tables) / 4); i += blockDim.x) dst[i] = __ldg(src + i);
  }
  const Tables* __restrict__ tab = kTabSmem<K> ? &tabs : tab_g;
  // the slot work of event e, its record already in rs (every thread of the block calls it)
  auto run_event = [&](const int64_t e) {
  __syncthreads();
  const bool active = slot < nslot;
  // groups past the last slot leave (every sync of the slot work is per group), except with the
  // tensor-core epilogue, whose MMAs take the whole warp: there they contribute zero jamps
  if (EPI != kMma && !active) return;
  SlotState<K, T>& S = sh[warp * GPW + grp];
  const int gc = active ? gslots[slot] : 0;   // bit g = helicity (+1) of gluon g
  auto ld = [&](int item) -> T { return rec_val(rs[item], static_cast<T*>(nullptr)); };
  const T gs = rec_val(static_cast<RecT>(cst.gs), static_cast<T*>(nullptr));
  // helicity index of (gc, top helicity, antitop helicity), and which of the four are in the mask
  int hbase = 0;
#pragma unroll
  for (int g = 0; g < K; ++g)
    if ((gc >> g) & 1) hbase |= 1 << (npar - 1 - (g < 2 ? g : g + 2));
  const int bit_t = 1 << (npar - 3), bit_tb = 1 << (npar - 4);
  bool good[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int h = hbase | ((k >> 1) ? bit_t : 0) | ((k & 1) ? bit_tb : 0);
    good[k] = active && ((mask[h >> 5] >> (h & 31)) & 1u);
  }
  if (active) {

    // ---- external gluon currents ----
    if (lane < K) {
      T pol[5];
#pragma unroll
      for (int i = 0; i < 5; ++i) pol[i] = ld(L::EPS + 5 * lane + i);
      cx<T> w[4];
      v2::ext_gluon(pol, (gc >> lane) & 1 ? 1 : -1, lane >= 2, w);
#pragma unroll
      for (int m = 0; m < 4; ++m) S.J[m][lane] = stw(w[m]);
    }
    __syncwarp(gmask);
    auto getJ = [&](int slot_ref, cx<T>* j) {
#pragma unroll
      for (int m = 0; m < 4; ++m) j[m] = ldw(S.J[m][slot_ref >> 1]);
    };
    auto getP = [&](int seq, T* P) {
      const int msk = tab->seq_mask[seq];
#pragma unroll
      for (int m = 0; m < 4; ++m) P[m] = ld(L::PT + 4 * msk + m);
    };
    // current of sequence s (splits from the tables) into acc
    auto current = [&](int nv3, const int16_t (*v3)[2], int nv4, const int16_t (*v4)[3], cx<T>* acc) {
      for (int k = 0; k < nv3; ++k) {
        const int rl = v3[k][0], rr = v3[k][1];
        cx<T> JL[4], JR[4];
        T PL[4], PR[4];
        getJ(rl, JL);
        getJ(rr, JR);
        getP(rl >> 1, PL);
        getP(rr >> 1, PR);
        v2::v3_acc(acc, JL, JR, PL, PR, ((rl ^ rr) & 1) != 0);
      }
      for (int k = 0; k < nv4; ++k) {
        const int ra = v4[k][0], rb = v4[k][1], rc = v4[k][2];
        cx<T> JA[4], JB[4], JC[4];
        getJ(ra, JA);
        getJ(rb, JB);
        getJ(rc, JC);
        v2::v4_acc(acc, JA, JB, JC, gs, ((ra ^ rb ^ rc) & 1) != 0);
      }
    };

    // ---- gluon currents by length: the sequences of one length are independent ----
#pragma unroll
    for (int len = 2; len < K; ++len) {
      for (int s = seq_start(K, len) + lane; s < seq_start(K, len + 1); s += G) {
        if constexpr (!DF && L::NPAIR > 0) {
          if (len == 2) {   // the pair's current from the FP32 record (FP64 arithmetic, record_j2)
            const int msk = tab->seq_mask[s];
            const int ga = __ffs(msk) - 1, gb = 31 - __clz(msk);
            const int h = ((gc >> ga) & 1) | (((gc >> gb) & 1) << 1);
            const float* it = static_cast<const float*>(rec_any) + (e / kPage) * L::NITEM * kPage + (e % kPage) +
                              (L::J2 + (v2::pair_index(K, ga, gb) * 4 + h) * 8) * kPage;
#pragma unroll
            for (int m = 0; m < 4; ++m) S.J[m][s] = stw(cx<T>{__ldg(it + 2 * m * kPage), __ldg(it + (2 * m + 1) * kPage)});
            continue;
          }
        }
        cx<T> acc[4] = {};
        current(tab->seq_nv3[s], tab->seq_v3[s], tab->seq_nv4[s], tab->seq_v4[s], acc);
        const T f = ld(L::GP + tab->seq_mask[s]);
#pragma unroll
        for (int m = 0; m < 4; ++m) S.J[m][s] = stw(v2::cscale(f, acc[m]));
      }
      __syncwarp(gmask);
    }
    // ---- all gluons on one current (canonical orderings) ----
    {
      const T fz = ld(L::GP + NSUB - 1);
      for (int f = lane; f < NFULL; f += G) {
        cx<T> acc[4] = {};
        current(tab->full_nv3[f], tab->full_v3[f], tab->full_nv4[f], tab->full_v4[f], acc);
#pragma unroll
        for (int m = 0; m < 4; ++m) S.JF[m][f] = stw(v2::cscale(fz, acc[m]));
      }
    }
    __syncwarp(gmask);

    // ---- quark line: half-group per top helicity, a run of orderings per lane ----
    {
      constexpr int H = G / 2;   // lanes per top helicity
      const int a = lane / H, hl = lane % H;
      const int c0 = hl * NCOL / H, c1 = (hl + 1) * NCOL / H;
      if (good[2 * a] || good[2 * a + 1]) {
        cx<T> vv[2][4], stk[K][4], Jq[2][4];
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int q = 0; q < 4; ++q) vv[b][q] = {ld(L::VV + (b * 4 + q) * 2), ld(L::VV + (b * 4 + q) * 2 + 1)};
#pragma unroll
        for (int q = 0; q < 4; ++q) stk[0][q] = {ld(L::UB + (a * 4 + q) * 2), ld(L::UB + (a * 4 + q) * 2 + 1)};
        v2::quark_current(stk[0], vv[0], Jq[0]);
        v2::quark_current(stk[0], vv[1], Jq[1]);
        for (int c = c0; c < c1; ++c) {
          const int l = c == c0 ? 0 : tab->lcp[c];
#pragma unroll
          for (int m = 1; m < K; ++m) {
            if (m <= l) continue;
            cx<T> acc[4] = {};
#pragma unroll
            for (int j = 0; j < m; ++j) {
              const int r = tab->sub[c][j][m];
              cx<T> Jr[4];
              getJ(r, Jr);
              v2::row_gamma_acc(acc, stk[j], Jr, (r & 1) != 0);
            }
            const int pm = tab->prefix_mask[c][m];
            T q[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) q[k] = ld(L::QC + 5 * pm + k);
            v2::row_prop(acc, q, stk[m]);
          }
          const int fi = tab->full_idx[c];
          const int fj = fi >= 0 ? fi : -fi - 1;
          const bool fneg = fi < 0 && !(K & 1);   // reflection sign (-1)^(K+1)
          cx<T> JFc[4];
#pragma unroll
          for (int m = 0; m < 4; ++m) JFc[m] = ldw(S.JF[m][fj]);
          cx<T> amp0 = v2::mdot(Jq[0], JFc), amp1 = v2::mdot(Jq[1], JFc);
          if (fneg) {
            amp0 = v2::cneg(amp0);
            amp1 = v2::cneg(amp1);
          }
#pragma unroll
          for (int j = 1; j < K; ++j) {
            const int r = tab->sub[c][j][K];
            cx<T> Jr[4], t[4] = {};
            getJ(r, Jr);
            v2::row_gamma_acc(t, stk[j], Jr, (r & 1) != 0);
            v2::sdot_acc(amp0, t, vv[0], false);
            v2::sdot_acc(amp1, t, vv[1], false);
          }
          S.A[2 * a][c] = good[2 * a] ? jamp32(amp0) : make_float2(0.f, 0.f);
          S.A[2 * a + 1][c] = good[2 * a + 1] ? jamp32(amp1) : make_float2(0.f, 0.f);
        }
      } else {
        for (int c = c0; c < c1; ++c) {
          S.A[2 * a][c] = make_float2(0.f, 0.f);
          S.A[2 * a + 1][c] = make_float2(0.f, 0.f);
        }
      }
    }
    __syncwarp(gmask);
  } else {   // a slot past the last one (tensor-core epilogue only): zero jamps
    for (int i = lane; i < 4 * NCOL; i += G) S.A[i / NCOL][i % NCOL] = make_float2(0.f, 0.f);
  }

  if constexpr (EPI == kJamps) {
    float2* row = jout + (e * (4 << K) + slot * 4) * NCOL;
    for (int i = lane; i < 4 * NCOL; i += G) row[i] = S.A[i / NCOL][i % NCOL];
  } else if constexpr (EPI == kSimt) {
    // colour sums of the four helicities at once: lane l forms rows x = l, l + G, ... of w_h = C A_h
    // (C symmetric: row y of C read along x, coalesced; each C value feeds 8 FMAs), then A_h^* . w_h
    // (real, imaginary) pairs on Blackwell's paired FP32 FMA: one instruction per colour-matrix entry
    // and helicity instead of two
    constexpr int XR = (NCOL + G - 1) / G;   // rows per lane
    uint64_t w2[4][XR];
#pragma unroll
    for (int h = 0; h < 4; ++h)
#pragma unroll
      for (int k = 0; k < XR; ++k) w2[h][k] = 0ull;
    for (int y = 0; y < NCOL; ++y) {
      uint64_t ay[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) ay[h] = pack2(S.A[h][y]);
#pragma unroll
      for (int k = 0; k < XR; ++k) {
        const int x = lane + G * k;
        const float cxy = x < NCOL ? __ldg(cfull + y * NCOL + x) : 0.f;
        const uint64_t cc = pack2(make_float2(cxy, cxy));
#pragma unroll
        for (int h = 0; h < 4; ++h) w2[h][k] = ffma2(cc, ay[h], w2[h][k]);
      }
    }
    float total = 0.f;   // summed in FP32 (these are FP32 colour sums), widened exactly at the end
#pragma unroll
    for (int h = 0; h < 4; ++h) {   // jamps of helicities outside the mask are zero: no branch needed
      uint64_t s2 = 0ull;
#pragma unroll
      for (int k = 0; k < XR; ++k) {
        const int x = lane + G * k;
        if (x < NCOL) s2 = ffma2(pack2(S.A[h][x]), w2[h][k], s2);
      }
      const float2 sp = unpack2(s2);
      float s = sp.x + sp.y;
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, G);
      if (good[h]) total += s;
    }
    if (lane == 0) {
      const double v = f32_times_pow2(total * static_cast<float>(cst.colour_scale), 0);
      if (rows_out) {   // tensor-core row layout (slot * 4 + helicity pair): the slot total in the first row
        out[(slot * 4) * stride + e] = v;
        out[(slot * 4 + 1) * stride + e] = 0.0;
        out[(slot * 4 + 2) * stride + e] = 0.0;
        out[(slot * 4 + 3) * stride + e] = 0.0;
      } else {
        out[slot * stride + e] = v;
      }
    }
  } else if constexpr (GPW == 1) {
    // colour sums on the tensor cores, one slot per warp (5 gluons): Y = C a for the slot's 8 vectors
    // a_n (helicity n/2, real part for even n, imaginary for odd) as D = C B, MMA rows = colour index x
    // (row-major A = C, exact FP16 integers), columns = the 8 vectors, k = colour index y, so every row
    // and column of every MMA is used.  Each vector is scaled by a power of two and split hi + lo 2^-11
    // in FP16 (B fragments, built once); FP32 accumulation; the quadratic form a_n . Y_n takes the FP32
    // jamps themselves.
    __syncwarp();
    if (!active) return;
    constexpr int KP = (NCOL + 15) / 16 * 16, KS = KP / 16, MT = KP / 16, LDH = KP + 8;
    static_assert(MT % 2 == 0, "row tiles in pairs");
    const int lw = threadIdx.x & 31, gq = lw >> 2, q = lw & 3;
    // B fragments of vector n = gq: k = 16 ks + 2q (+1) and + 8 (+9)
    const float2* av = S.A[gq >> 1];
    const bool im = gq & 1;
    auto comp = [&](int y) -> float {
      if (y >= NCOL) return 0.f;
      const float2 v = av[y];
      return im ? v.y : v.x;
    };
    float mx = 0.f;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks)
#pragma unroll
      for (int j = 0; j < 4; ++j) mx = fmaxf(mx, fabsf(comp(ks * 16 + 2 * q + (j & 1) + (j >> 1) * 8)));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    int ex = 0;
    if (mx > 0.f) frexpf(mx, &ex);
    const float sc = ldexpf(1.f, -ex);
    uint32_t bh[KS][2], bl[KS][2];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks)
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int y = ks * 16 + 2 * q + 8 * half;
        const float x0 = comp(y) * sc, x1 = comp(y + 1) * sc;
        const __half h0 = __float2half_rn(x0), h1 = __float2half_rn(x1);
        const __half l0 = __float2half_rn((x0 - __half2float(h0)) * 2048.f);
        const __half l1 = __float2half_rn((x1 - __half2float(h1)) * 2048.f);
        bh[ks][half] = pack_h2(h0, h1);
        bl[ks][half] = pack_h2(l0, l1);
      }
    // this thread's D columns are vectors 2q (real part) and 2q + 1 (imaginary part) of helicity q, at
    // rows x = 16 mt + gq and + 8
    const float2* aq = S.A[q];
    float sr = 0.f, si = 0.f;
    const unsigned int* cw = reinterpret_cast<const unsigned int*>(cmat16);
#pragma unroll
    for (int mt = 0; mt < MT; mt += 2) {
      float dh[2][4] = {}, dl[2][4] = {};
#pragma unroll
      for (int ks = 0; ks < KS; ++ks)
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int x0 = (mt + u) * 16 + gq, y0 = ks * 16 + 2 * q;
          uint32_t af[4];
          af[0] = x0 < NCOL ? __ldg(cw + (x0 * LDH + y0) / 2) : 0u;
          af[1] = x0 + 8 < NCOL ? __ldg(cw + ((x0 + 8) * LDH + y0) / 2) : 0u;
          af[2] = x0 < NCOL ? __ldg(cw + (x0 * LDH + y0 + 8) / 2) : 0u;
          af[3] = x0 + 8 < NCOL ? __ldg(cw + ((x0 + 8) * LDH + y0 + 8) / 2) : 0u;
          mma16816(dh[u], af, bh[ks]);
          mma16816(dl[u], af, bl[ks]);
        }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int x = (mt + u) * 16 + gq + 8 * r;
          if (x < NCOL) {
            const float2 a = aq[x];
            sr = fmaf(a.x, fmaf(dl[u][2 * r], 1.f / 2048.f, dh[u][2 * r]), sr);
            si = fmaf(a.y, fmaf(dl[u][2 * r + 1], 1.f / 2048.f, dh[u][2 * r + 1]), si);
          }
        }
    }
    // sum over the rows (lanes with the same q), undo the vector scales (exact powers of two: the
    // exponent of vector n sits in lanes 4n .. 4n + 3), then sum the four helicities
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    const int exr = __shfl_sync(0xffffffffu, ex, 8 * q), exi = __shfl_sync(0xffffffffu, ex, 8 * q + 4);
    double v = static_cast<double>(sr) * pow2d(exr) + static_cast<double>(si) * pow2d(exi);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    if (lw == 0) out[slot * stride + e] = v * cst.colour_scale;
  } else {
    // colour sums on the tensor cores, the warp's slots together: MMA rows = (slot, helicity, Re/Im),
    // 8 per slot; each row scaled by a power of two and split hi + lo 2^-11 in FP16 against the exact
    // FP16 integer colour matrix, FP32 accumulation (as the separate tensor-core colour kernel)
    __syncwarp();
    constexpr int KP = (NCOL + 15) / 16 * 16, KS = KP / 16, NT = (NCOL + 7) / 8, LDH = KP + 8;
    constexpr int ROWS = 8 * GPW, MT = (ROWS + 15) / 16;
    const int lw = threadIdx.x & 31, gq = lw >> 2, q = lw & 3;
    const SlotState<K>* SW = &sh[warp * GPW];
    auto elem = [&](int r, int c) -> float {
      if (r >= ROWS || c >= NCOL) return 0.f;
      const float2 v = SW[r >> 3].A[(r & 7) >> 1][c];
      return (r & 1) ? v.y : v.x;
    };
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      const int r0 = 16 * t + gq, r1 = r0 + 8;
      float m0 = 0.f, m1 = 0.f;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = ks * 16 + 2 * q + (j & 1) + (j >> 1) * 8;
          m0 = fmaxf(m0, fabsf(elem(r0, c)));
          m1 = fmaxf(m1, fabsf(elem(r1, c)));
        }
      m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 1));
      m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 2));
      m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 1));
      m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 2));
      int ex0 = 0, ex1 = 0;
      if (m0 > 0.f) frexpf(m0, &ex0);
      if (m1 > 0.f) frexpf(m1, &ex1);
      const float sc0 = ldexpf(1.f, -ex0), sc1 = ldexpf(1.f, -ex1);
      uint32_t ah[KS][4], al[KS][4];
#pragma unroll
      for (int ks = 0; ks < KS; ++ks)
#pragma unroll
        for (int rg = 0; rg < 4; ++rg) {
          const int c = ks * 16 + 2 * q + (rg >> 1) * 8;
          const int r = (rg & 1) ? r1 : r0;
          const float sc = (rg & 1) ? sc1 : sc0;
          const float x0 = elem(r, c) * sc, x1 = elem(r, c + 1) * sc;
          const __half h0 = __float2half_rn(x0), h1 = __float2half_rn(x1);
          const __half l0 = __float2half_rn((x0 - __half2float(h0)) * 2048.f);
          const __half l1 = __float2half_rn((x1 - __half2float(h1)) * 2048.f);
          ah[ks][rg] = pack_h2(h0, h1);
          al[ks][rg] = pack_h2(l0, l1);
        }
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        float dh[4] = {0.f, 0.f, 0.f, 0.f}, dl[4] = {0.f, 0.f, 0.f, 0.f};
        const __half* cb = cmat16 + (nt * 8 + gq) * LDH + 2 * q;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
          uint32_t bf[2];
          bf[0] = __ldg(reinterpret_cast<const unsigned int*>(cb + ks * 16));
          bf[1] = __ldg(reinterpret_cast<const unsigned int*>(cb + ks * 16 + 8));
          mma16816(dh, ah[ks], bf);
          mma16816(dl, al[ks], bf);
        }
        // this thread's Y columns nt*8 + 2q, +1 are the a columns it holds in k step nt/2, half nt%2
        const int ksa = nt >> 1, hb = (nt & 1) * 2;
        const float r = 1.f / 2048.f;
        s0 = fmaf(unsplit(ah[ksa][hb], al[ksa][hb], 0), fmaf(dl[0], r, dh[0]), s0);
        s0 = fmaf(unsplit(ah[ksa][hb], al[ksa][hb], 1), fmaf(dl[1], r, dh[1]), s0);
        s1 = fmaf(unsplit(ah[ksa][hb + 1], al[ksa][hb + 1], 0), fmaf(dl[2], r, dh[2]), s1);
        s1 = fmaf(unsplit(ah[ksa][hb + 1], al[ksa][hb + 1], 1), fmaf(dl[3], r, dh[3]), s1);
      }
      s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
      s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
      s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
      s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
      // sum the 8 rows of a slot (rows gq = 0..7 sit in lanes 4 gq) in FP32 at the largest exponent of
      // its nonzero rows (C is positive definite: a row's sum is 0 only for a zero row), then widen
      // exactly to FP64 (no FP64 instruction: that pipe runs at 1/64 of the FP32 rate)
      constexpr int kNone = -100000;
      int E0 = s0 != 0.f ? 2 * ex0 : kNone, E1 = s1 != 0.f ? 2 * ex1 : kNone;
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        E0 = max(E0, __shfl_xor_sync(0xffffffffu, E0, o));
        E1 = max(E1, __shfl_xor_sync(0xffffffffu, E1, o));
      }
      float u0 = s0 != 0.f ? s0 * pow2f_neg(2 * ex0 - E0) : 0.f;
      float u1 = s1 != 0.f ? s1 * pow2f_neg(2 * ex1 - E1) : 0.f;
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        u0 += __shfl_xor_sync(0xffffffffu, u0, o);
        u1 += __shfl_xor_sync(0xffffffffu, u1, o);
      }
      if (lw == 0) {
        const float csf = static_cast<float>(cst.colour_scale);
        const int sa = 2 * t, sb = 2 * t + 1;   // the slots of rows 0-7 and 8-15 of this tile
        if (sa < GPW && slot0 + sa < nslot) out[(slot0 + sa) * stride + e] = f32_times_pow2(u0 * csf, E0);
        if (sb < GPW && slot0 + sb < nslot) out[(slot0 + sb) * stride + e] = f32_times_pow2(u1 * csf, E1);
      }
    }
  }
  };   // run_event

  if constexpr (!DF) {
    const int64_t e = blockIdx.x;   // one block per event: e < nevt
    if (skip && skip[e]) return;    // recomputed by another launch (the whole block: one event)
    const float* in = static_cast<const float*>(rec_any) + (e / kPage) * L::NITEM * kPage + (e % kPage);
    for (int i = threadIdx.x; i < L::NBASE; i += blockDim.x) rs[i] = __ldg(in + i * kPage);
    run_event(e);
  } else {
    const double* mom = static_cast<const double*>(rec_any);
    const int n = *nlist;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
      const int64_t e = evlist[i];
      __syncthreads();   // the previous event's slot work has finished reading the record
      if ((threadIdx.x & 31) == 0) {   // one part of the FP64 record per warp
        double p[npar][4];
        const double* base = mom + (e / kPage) * npar * 4 * kPage + (e % kPage);
#pragma unroll
        for (int q = 0; q < npar; ++q)
#pragma unroll
          for (int m = 0; m < 4; ++m) p[q][m] = __ldg(base + (q * 4 + m) * kPage);
        auto put = [&](int item, double v) { rs[item] = v; };
        if (warp == 0) v2::record_subsets<K, double, 0, NSUB / 2>(p, cst, put);
        else if (warp == 1) v2::record_subsets<K, double, NSUB / 2, NSUB>(p, cst, put);
        else if (warp == 2) v2::record_pols<K, double>(p, put);
        else v2::record_tops<K, double>(p, cst, put);
      }
      run_event(e);
    }
  }

}

template <int K>
static cudaError_t launch_k(const void* rec, int64_t nevt, const Tables* tab, const int* gslots, int maxslot,
                            const int* nslot, const uint32_t* mask, const float* cfull, const void* cmat16, int epi,
                            const MeConst& cst, double* out, int64_t stride, float2* jout, const uint8_t* skip,
                            cudaStream_t st) {
  if (nevt <= 0 || maxslot <= 0) return cudaSuccess;
  if (nevt > 0x7fffffffLL) return cudaErrorInvalidValue;
  constexpr int per_block = kWarps * (32 / WSizes<K>::G);   // slots per block
  const dim3 grid(static_cast<unsigned>(nevt), static_cast<unsigned>((maxslot + per_block - 1) / per_block));
  const float* r = static_cast<const float*>(rec);
  const __half* c16 = static_cast<const __half*>(cmat16);
  constexpr size_t smem = SmemLayout<K>::bytes;
  // opt in to more than 48 KB of dynamic shared memory, once per device (a bit per device; racing
  // first calls both set it)
  static std::atomic<unsigned long long> configured{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(configured.load(std::memory_order_acquire) & bit)) {
    cudaError_t e = cudaFuncSetAttribute(k_me_warp<K, kJamps>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_me_warp<K, kMma>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_me_warp<K, kSimt>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    configured.fetch_or(bit, std::memory_order_release);
  }
  if (epi == kJamps)
    { k_me_warp<K, kJamps><<<grid, kWarps * 32, smem, st>>>(r, nevt, tab, gslots, nslot, mask, cfull, c16, cst, out,
                                                          stride, jout, skip); mg::note_launch(); }
  else if (epi == kMma)
    { k_me_warp<K, kMma><<<grid, kWarps * 32, smem, st>>>(r, nevt, tab, gslots, nslot, mask, cfull, c16, cst, out, stride,
                                                        nullptr, skip); mg::note_launch(); }
  else
    { k_me_warp<K, kSimt><<<grid, kWarps * 32, smem, st>>>(r, nevt, tab, gslots, nslot, mask, cfull, c16, cst, out,
                                                         stride, nullptr, skip); mg::note_launch(); }
  return cudaGetLastError();
}

template <int K>
static cudaError_t launch_dd_k(const double* mom, int64_t nevt, const Tables* tab, const int* gslots, int maxslot,
                               const int* nslot, const uint32_t* mask, const float* cfull, const MeConst& cst,
                               double* out, int64_t stride, const int* evlist, const int* nlist, int rows_out,
                               cudaStream_t st) {
  if (nevt <= 0 || maxslot <= 0) return cudaSuccess;
  constexpr int per_block = kWarps * (32 / WSizes<K>::G);   // slots per block
  // the blocks walk the list with a stride of gridDim.x (its length is known on the device only)
  const unsigned gx = static_cast<unsigned>(nevt < 2048 ? nevt : 2048);
  const dim3 grid(gx, static_cast<unsigned>((maxslot + per_block - 1) / per_block));
  constexpr size_t smem = SmemLayout<K, dd::df>::bytes;
  static std::atomic<unsigned long long> configured{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(configured.load(std::memory_order_acquire) & bit)) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_me_warp<K, kSimt, dd::df>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    configured.fetch_or(bit, std::memory_order_release);
  }
  { k_me_warp<K, kSimt, dd::df><<<grid, kWarps * 32, smem, st>>>(mom, nevt, tab, gslots, nslot, mask, cfull, nullptr, cst,
                                                                out, stride, nullptr, nullptr, evlist, nlist, rows_out);
    mg::note_launch(); }
  return cudaGetLastError();
}

}  // namespace wk

bool me_warp_available(int K, bool fp32) { return fp32 && K >= 3 && K <= 5; }

cudaError_t launch_me_warp(int K, const void* rec, int64_t nevt, const Tables* tab, const int* gslots, int maxslot,
                           const int* nslot, const uint32_t* mask, const float* cfull, const void* cmat16, int epi,
                           const MeConst& cst, double* out, int64_t stride, float2* jout, const uint8_t* skip,
                           cudaStream_t st) {
  switch (K) {
    case 3: return wk::launch_k<3>(rec, nevt, tab, gslots, maxslot, nslot, mask, cfull, cmat16, epi, cst, out, stride, jout, skip, st);
    case 4: return wk::launch_k<4>(rec, nevt, tab, gslots, maxslot, nslot, mask, cfull, cmat16, epi, cst, out, stride, jout, skip, st);
    case 5: return wk::launch_k<5>(rec, nevt, tab, gslots, maxslot, nslot, mask, cfull, cmat16, epi, cst, out, stride, jout, skip, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_me_warp_repair(int K, const double* mom, int64_t nevt, const Tables* tab, const int* gslots,
                                  int maxslot, const int* nslot, const uint32_t* mask, const float* cfull,
                                  const MeConst& cst, double* out, int64_t stride, const int* evlist, const int* nlist,
                                  int rows_out, cudaStream_t st) {
  switch (K) {
    case 3: return wk::launch_dd_k<3>(mom, nevt, tab, gslots, maxslot, nslot, mask, cfull, cst, out, stride, evlist, nlist, rows_out, st);
    case 4: return wk::launch_dd_k<4>(mom, nevt, tab, gslots, maxslot, nslot, mask, cfull, cst, out, stride, evlist, nlist, rows_out, st);
    case 5: return wk::launch_dd_k<5>(mom, nevt, tab, gslots, maxslot, nslot, mask, cfull, cst, out, stride, evlist, nlist, rows_out, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mg
