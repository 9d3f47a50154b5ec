// mg_colour_tc.cu -- colour sum A^dagger C A on the tensor cores.
//
// Colour decomposition (Mangano-Parke): sum over colours of |M_h|^2 = Re(A)^T C Re(A) + Im(A)^T C Im(A)
// with the exact colour matrix C = Cint / den.  Viewed over all (event, helicity) pairs this is a
// dense (2 nevt nhel) x ncol x ncol contraction, run here with mma.sync m16n8k16 (f16 x f16 -> f32):
//   * Cint is held exactly in FP16 (every entry is an integer <= 2048 or a power of two: max 4096
//     for 120 colour flows);
//   * every row (the real or the imaginary part of one jamp vector) is scaled by a power of two to
//     max |a| in [1/2, 1) and split a = hi + lo 2^-11 with hi, lo FP16, so a is carried to ~22 bits;
//   * Y = C a is accumulated in FP32 (two accumulators, hi and lo), and the row's quadratic form
//     a . Y is formed in FP32 with a = hi + lo 2^-11, then unscaled exactly;
//   * each warp stages its next tile of jamp vectors into shared memory with cp.async while it computes
//     the current one, whose A fragments are built once in registers for all column tiles.
// Relative error per (event, helicity) ~1e-7 (the colour matrices are well conditioned: kappa <= 16).
// Rows: jamps[(e * rows_alloc + r) * ncol + sigma] (FP32 complex), r < *nrows_dev; output:
// out[r * stride + e] = colour sum * scale, in FP64.  rows_alloc is a power of two (the helicity count),
// so the kernel walks the padded row index q = e * rows_alloc + r with shifts and masks: a tile of 8
// consecutive q is 8 rows of one event, and rows r >= *nrows_dev are zero-filled, never read.
#include <atomic>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "mg_alloc.h"
#include "mg_internal.h"
#include "mg_kernels.h"

namespace mg {
namespace {

// 2^k as a float from its exponent bits (exact), 0 below the normal range; k <= 0 here
__device__ __forceinline__ float pow2f_neg(int k) {
  return k >= -126 ? __uint_as_float(static_cast<unsigned>(127 + k) << 23) : 0.f;
}

// s 2^E as a double, built from the IEEE 754 fields of the float s (exact: the mantissa is copied and
// the exponent moved).  No FP64 instruction for normal s: the FP64 pipe is 1/64 of the FP32 one, and
// this kernel's epilogue would otherwise spend most of its time there.  Zero and FP32 subnormals (never
// seen for these colour sums) take the FP64 route.
__device__ __forceinline__ double f32_times_pow2(float s, int E) {
  const unsigned u = __float_as_uint(s);
  const unsigned ef = (u >> 23) & 0xffu;
  if ((u & 0x7fffffffu) == 0) return 0.0;   // E may be a placeholder here
  if (ef == 0) return static_cast<double>(s) * __longlong_as_double(static_cast<long long>(1023 + E) << 52);
  const unsigned long long bits = (static_cast<unsigned long long>(u >> 31) << 63) |
                                  (static_cast<unsigned long long>(static_cast<int>(ef) - 127 + E + 1023) << 52) |
                                  (static_cast<unsigned long long>(u & 0x7fffffu) << 29);
  return __longlong_as_double(static_cast<long long>(bits));
}

// (a 2^ea + b 2^eb) scale: the colour sums of a vector's real and imaginary rows, each under its own
// power-of-two row scale; summed in FP32 at the larger exponent of the nonzero rows (C is positive
// definite, so a row's sum is 0 only for a zero row, whose exponent means nothing), then widened exactly
__device__ __forceinline__ double combine_rows(float a, int ea, float b, int eb, float scale) {
  if (a == 0.f) return f32_times_pow2(b * scale, eb);
  if (b == 0.f) return f32_times_pow2(a * scale, ea);
  const int E = ea > eb ? ea : eb;
  const float t = fmaf(a, pow2f_neg(ea - E), b * pow2f_neg(eb - E)) * scale;
  return f32_times_pow2(t, E);
}

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int NCOL>
struct TcShape {
  static constexpr int KP = (NCOL + 15) / 16 * 16;   // contraction length, padded to the MMA k
  static constexpr int KS = KP / 16;                 // MMA k steps
  static constexpr int NT = (NCOL + 7) / 8;          // output column tiles of 8
  static constexpr int NP = NT * 8;
  static constexpr int LDH = KP + 8;                 // half pitch of C (breaks bank conflicts)
  static constexpr int WARPS = 4;
  static constexpr int CHUNKS = 8 * NCOL / 2;        // 16-byte pieces of one tile (8 jamp vectors)
  static constexpr size_t c_bytes() { return sizeof(__half) * size_t(NP) * LDH; }
  static constexpr size_t smem_bytes() { return c_bytes() + sizeof(float2) * size_t(WARPS) * 2 * 8 * NCOL; }
};

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src, bool valid) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst_smem));
  const int n = valid ? 16 : 0;   // 0: nothing is read, the 16 bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_h2(__half lo_half, __half hi_half) {
  return static_cast<uint32_t>(__half_as_ushort(lo_half)) | (static_cast<uint32_t>(__half_as_ushort(hi_half)) << 16);
}

// hi/lo FP16 split of a scaled value t: t ~ hi + lo 2^-11
__device__ __forceinline__ void split_h(float t, __half& hi, __half& lo) {
  hi = __float2half_rn(t);
  lo = __float2half_rn((t - __half2float(hi)) * 2048.f);
}

// value of the FP16 pair element k (0 low, 1 high) of a hi/lo split, as FP32
__device__ __forceinline__ float unsplit(uint32_t h, uint32_t l, int k) {
  const __half hh = __ushort_as_half(static_cast<unsigned short>(k ? h >> 16 : h & 0xffffu));
  const __half lh = __ushort_as_half(static_cast<unsigned short>(k ? l >> 16 : l & 0xffffu));
  return fmaf(__half2float(lh), 1.f / 2048.f, __half2float(hh));
}

// One warp per tile of 8 (event, helicity) jamp vectors = 16 MMA rows (row 2p: Re, 2p+1: Im of vector p),
// tiles strided over the grid.  The next tile is staged into shared memory with cp.async while the
// current one is computed; the current tile's A fragments (hi and lo) are built once, in registers, and
// serve every column tile of Y = C a and the row's quadratic form a . Y.
template <int NCOL>
__global__ void __launch_bounds__(128) k_colour_tc(const float2* __restrict__ jamps, int64_t nevt, int rows_log2,
                                                   const int* __restrict__ nrows_dev, const __half* __restrict__ cmat,
                                                   double scale, double* __restrict__ out, int64_t stride,
                                                   const uint8_t* __restrict__ skip) {
  using S = TcShape<NCOL>;
  constexpr int KS = S::KS, NT = S::NT, NP = S::NP, LDH = S::LDH;
  extern __shared__ __align__(16) unsigned char smem[];
  __half* sC = reinterpret_cast<__half*>(smem);                       // [NP][LDH]: C[n][k]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* sRaw = reinterpret_cast<float2*>(smem + S::c_bytes()) + warp * 2 * 8 * NCOL;   // [2][8][NCOL]

  for (int i = threadIdx.x; i < NP * LDH; i += blockDim.x) sC[i] = cmat[i];
  __syncthreads();

  const float scale_f = static_cast<float>(scale);
  const int nrows = *nrows_dev;
  const int64_t rmask = (int64_t(1) << rows_log2) - 1;
  const int64_t ntiles = ((nevt << rows_log2) + 7) / 8;
  const int64_t tstep = static_cast<int64_t>(gridDim.x) * S::WARPS;
  const int g = lane >> 2, q = lane & 3;

  auto stage = [&](int64_t tile, int buf) {
    float2* dst = sRaw + buf * 8 * NCOL;
    for (int i = lane; i < S::CHUNKS; i += 32) {
      const int p = i / (NCOL / 2), w = i - p * (NCOL / 2);
      const int64_t qq = tile * 8 + p;
      const float2* src = jamps;
      bool valid = false;
      if (tile < ntiles) {
        const int64_t e = qq >> rows_log2;
        // rows past the last good one, and skipped events: no jamps (zeros)
        valid = (qq & rmask) < nrows && (!skip || !skip[e]);
        src = jamps + qq * NCOL + 2 * w;
      }
      cp_async16(dst + p * NCOL + 2 * w, src, valid);
    }
    cp_async_commit();
  };

  int64_t tile = static_cast<int64_t>(blockIdx.x) * S::WARPS + warp;
  int buf = 0;
  if (tile < ntiles) stage(tile, 0);
  for (; tile < ntiles; tile += tstep, buf ^= 1) {
    stage(tile + tstep, buf ^ 1);   // next tile (an empty group past the end)
    cp_async_wait1();
    __syncwarp();
    const float2* raw = sRaw + buf * 8 * NCOL;
    // rows g and g + 8 of the MMA tile: vectors g/2 and g/2 + 4, real (g even) or imaginary part
    const float2* v0 = raw + (g >> 1) * NCOL;
    const float2* v1 = raw + ((g >> 1) + 4) * NCOL;
    const bool im = g & 1;
    auto elem = [&](const float2* v, int c) -> float {
      if (c >= NCOL) return 0.f;
      const float2 x = v[c];
      return im ? x.y : x.x;
    };
    // per-row power-of-two scale: max |a| over the row (4 lanes of a quad hold it)
    float m0 = 0.f, m1 = 0.f;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = ks * 16 + 2 * q + (j & 1) + (j >> 1) * 8;
        m0 = fmaxf(m0, fabsf(elem(v0, c)));
        m1 = fmaxf(m1, fabsf(elem(v1, c)));
      }
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 1));
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 2));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 1));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 2));
    int ex0 = 0, ex1 = 0;
    if (m0 > 0.f) frexpf(m0, &ex0);
    if (m1 > 0.f) frexpf(m1, &ex1);
    const float sc0 = ldexpf(1.f, -ex0), sc1 = ldexpf(1.f, -ex1);
    // A fragments (m16n8k16, row-major A): regs 0/1 rows g / g+8 at k = 2q, 2q+1; regs 2/3 at k + 8
    uint32_t ah[KS][4], al[KS][4];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks)
#pragma unroll
      for (int rg = 0; rg < 4; ++rg) {
        const int c = ks * 16 + 2 * q + (rg >> 1) * 8;
        const float2* v = (rg & 1) ? v1 : v0;
        const float sc = (rg & 1) ? sc1 : sc0;
        __half h0, l0, h1, l1;
        split_h(elem(v, c) * sc, h0, l0);
        split_h(elem(v, c + 1) * sc, h1, l1);
        ah[ks][rg] = pack_h2(h0, h1);
        al[ks][rg] = pack_h2(l0, l1);
      }
    __syncwarp();   // this buffer is staged again two tiles later
    // Y = C a, two column tiles at a time (four independent accumulator chains); the quadratic form
    // a . Y of rows g and g + 8
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int n0 = 0; n0 < NT; n0 += 2) {
      constexpr int W = 2;
      float dh[W][4] = {}, dl[W][4] = {};
#pragma unroll
      for (int ks = 0; ks < KS; ++ks)
#pragma unroll
        for (int j = 0; j < W; ++j) {
          if (n0 + j >= NT) continue;
          const __half* cb = sC + ((n0 + j) * 8 + g) * LDH + 2 * q + ks * 16;
          uint32_t bf[2];
          bf[0] = *reinterpret_cast<const uint32_t*>(cb);
          bf[1] = *reinterpret_cast<const uint32_t*>(cb + 8);
          mma16816(dh[j], ah[ks], bf);
          mma16816(dl[j], al[ks], bf);
        }
#pragma unroll
      for (int j = 0; j < W; ++j) {
        const int nt = n0 + j;
        if (nt >= NT) continue;
        // this thread's Y columns nt*8 + 2q, +1 are the a columns it holds in k step nt/2, half nt%2
        const int ksa = nt >> 1, hb = (nt & 1) * 2;
        const float r = 1.f / 2048.f;
        s0 = fmaf(unsplit(ah[ksa][hb], al[ksa][hb], 0), fmaf(dl[j][0], r, dh[j][0]), s0);
        s0 = fmaf(unsplit(ah[ksa][hb], al[ksa][hb], 1), fmaf(dl[j][1], r, dh[j][1]), s0);
        s1 = fmaf(unsplit(ah[ksa][hb + 1], al[ksa][hb + 1], 0), fmaf(dl[j][2], r, dh[j][2]), s1);
        s1 = fmaf(unsplit(ah[ksa][hb + 1], al[ksa][hb + 1], 1), fmaf(dl[j][3], r, dh[j][3]), s1);
      }
    }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    // the real and imaginary rows of a vector sit in quads g and g^1 (lanes 4 apart): their sums and
    // row exponents, combined in the writing lanes
    const float t0 = __shfl_xor_sync(0xffffffffu, s0, 4), t1 = __shfl_xor_sync(0xffffffffu, s1, 4);
    const int f0 = __shfl_xor_sync(0xffffffffu, ex0, 4), f1 = __shfl_xor_sync(0xffffffffu, ex1, 4);
    if (q == 0 && (g & 1) == 0) {
      const int64_t qa = tile * 8 + g / 2, qb = tile * 8 + 4 + g / 2;
      const int64_t e = qa >> rows_log2;   // the tile's 8 rows belong to one event
      if (!skip || !skip[e]) {
        if ((qa & rmask) < nrows) out[(qa & rmask) * stride + e] = combine_rows(s0, 2 * ex0, t0, 2 * f0, scale_f);
        if ((qb & rmask) < nrows) out[(qb & rmask) * stride + e] = combine_rows(s1, 2 * ex1, t1, 2 * f1, scale_f);
      }
    }
  }
  cp_async_wait0();
}

template <int NCOL>
cudaError_t launch_tc(const float2* jamps, int64_t nevt, int rows_alloc, const int* nrows, const __half* cmat,
                      double scale, double* out, int64_t stride, const uint8_t* skip, cudaStream_t st) {
  using S = TcShape<NCOL>;
  int rows_log2 = 0;   // rows_alloc: a power of two, at least one tile (8 rows)
  while ((1 << rows_log2) < rows_alloc) ++rows_log2;
  if ((1 << rows_log2) != rows_alloc || rows_alloc < 8) return cudaErrorInvalidValue;
  const size_t smem = S::smem_bytes();
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  // the shared-memory opt-in, once per device (a bit per device; racing first calls both set it)
  static std::atomic<unsigned long long> configured{0};
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(configured.load(std::memory_order_acquire) & bit)) {
    cudaError_t e = cudaFuncSetAttribute(k_colour_tc<NCOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    configured.fetch_or(bit, std::memory_order_release);
  }
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_colour_tc<NCOL>, 128, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int64_t tiles = (nevt * rows_alloc + 7) / 8;
  int64_t blocks = (tiles + S::WARPS - 1) / S::WARPS;
  const int64_t cap = static_cast<int64_t>(nsm) * per_sm;   // resident blocks; tiles are strided over them
  if (blocks > cap) blocks = cap;
  if (blocks < 1) return cudaSuccess;
  { k_colour_tc<NCOL><<<static_cast<unsigned>(blocks), 128, smem, st>>>(jamps, nevt, rows_log2, nrows, cmat, scale, out,
                                                                       stride, skip); mg::note_launch(); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------------
// The same colour sums on the fifth-generation tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// One persistent CTA of 8 warps per SM walks "stages" of VECS = 64 S jamp vectors (128 S real rows, S
// M=128 MMA tiles; S NP = 128 accumulator columns in TMEM, NP = the padded colour count).  Per stage:
//   1. the stage's FP32 jamps, prefetched into registers with coalesced 16-byte loads during the previous
//      stage, go to a padded staging buffer in shared memory (row pitch 2 NCOL + 2 floats: the per-row
//      reads below are free of bank conflicts);
//   2. each row (real or imaginary part of one vector) is scaled by a power of two to max |t| in
//      [1/2, 1) and split t = hi + lo (two FP16 values, lo = fp16(t - hi) keeps t to ~2^-24 absolute),
//      written as the MMA's A operand in the no-swizzle K-major layout (8-row x 16-byte core matrices,
//      k-chunks 128 bytes apart, 8-row groups 16 (K/8) + 16 bytes apart: the extra 16 bytes spread the
//      16-byte stores of the 32 lanes, each a different vector, evenly over the banks);
//   3. one thread issues S x (K/16) x 2 MMAs (M = 128, N = NP, K = 16; hi, then lo, into the same FP32
//      accumulator: Y = C hi + C lo) against the exact integer colour matrix C (FP16, resident in shared
//      memory for the whole kernel) and commits them to the stage's mbarrier;
//   4. meanwhile the 8 warps finish the PREVIOUS stage (A and the accumulators are double-buffered):
//      they read its Y back (tcgen05.ld, warp w: TMEM lanes 32 (w % 4) .. +31, one half of the columns)
//      and form each row's quadratic form t . Y with t = hi + lo from its A buffer; the real and
//      imaginary rows of a vector are combined and unscaled exactly, as in k_colour_tc.
// Every wait is bounded: a wait that gives up records the stage in *err, and the CTA frees its tensor
// memory and returns.
template <int NCOL>
struct Umma {
  static constexpr int KP = (NCOL + 15) / 16 * 16;   // contraction length padded to the MMA K
  static constexpr int NP = KP;                       // C is square: N = K (a multiple of 16)
  static constexpr int S = 128 / NP;                  // MMA tiles per stage: S NP = 128 TMEM columns
  static constexpr int ROWS = 128 * S;
  static constexpr int VECS = ROWS / 2;
  static constexpr int PITCH = 2 * NCOL + 2;          // staging floats per vector
  static constexpr int CH = (NCOL + 7) / 8;           // 8-element k chunks holding data
  static constexpr int KC = KP / 8;                   // k chunks per row, padding included
  static constexpr int SBO_A = KC * 128 + 16;         // bytes between 8-row groups of A
  static constexpr int SBO_B = KC * 128;              // bytes between 8-row groups of B = C
  static constexpr int A_BYTES = (ROWS / 8) * SBO_A;  // one of hi / lo
  static constexpr int B_BYTES = (NP / 8) * SBO_B;
  static constexpr int STG_BYTES = VECS * PITCH * 4;
  static constexpr int F4 = VECS * NCOL * 2 / 4;      // 16-byte pieces of a stage
  static constexpr int THREADS = 256;
  static constexpr int PF = (F4 + THREADS - 1) / THREADS;   // prefetched pieces per thread
  static constexpr int VPL = CH <= 4 ? 32 : 8;        // vectors per warp in the conversion
  static constexpr int CPL = VPL == 32 ? CH : (CH + 3) / 4;   // k chunks per lane
  static constexpr int PASSES = VECS / (8 * VPL);
  static constexpr int CHALF = S == 1 ? (CH + 1) / 2 : 0;     // S = 1: data chunks of the first column half
  // shared memory (128-byte aligned pieces): A hi, lo for two buffers | B | staging | partial sums
  // [2][S][128] | row exponents [2][S][128] | 2 mbarriers, TMEM address, abort flag
  static constexpr int A_PAD = (A_BYTES + 127) / 128 * 128;
  static constexpr int OFF_B = 4 * A_PAD;
  static constexpr int OFF_STG = OFF_B + (B_BYTES + 127) / 128 * 128;
  static constexpr int OFF_PART = OFF_STG + (STG_BYTES + 127) / 128 * 128;
  static constexpr int OFF_EXP = OFF_PART + 2 * S * 128 * 4;
  static constexpr int OFF_VAL = OFF_EXP + 2 * S * 128 * 4;
  static constexpr int OFF_BAR = OFF_VAL + (2 * VECS + 127) / 128 * 128;
  static constexpr int VPT = (VECS + THREADS - 1) / THREADS;   // vector validity flags prefetched per thread
  static constexpr int SMEM = OFF_BAR + 64 + 128;     // + 128: the dynamic buffer is aligned up to 128 bytes
  static constexpr uint32_t IDESC = (1u << 4) | (static_cast<uint32_t>(NP >> 3) << 17) | (static_cast<uint32_t>(128 >> 4) << 24);
  static_assert(S * NP == 128 && PASSES * 8 * VPL == VECS && (2 * NCOL) % 4 == 0, "stage shape");
  static_assert(SMEM <= 232448, "shared memory");
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor, no swizzle: start, leading (k-chunk) and stride (8-row group) byte offsets
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(lbo >> 4) << 16) |
         (static_cast<uint64_t>(sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// FP16x2 hi and lo words of the value pair (a, b), |a|, |b| < 1: hi = fp16(a), fp16(b); lo = fp16 of
// the remainders (exact in FP32)
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hw, uint32_t& lw) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
  hw = *reinterpret_cast<const uint32_t*>(&h);
  lw = *reinterpret_cast<const uint32_t*>(&l);
}

// t . y over 8 k values: t = hi + lo from the 16-byte hi and lo chunks, y from the accumulator columns
__device__ __forceinline__ float dot8(uint4 h, uint4 l, const uint32_t* y, float acc) {
  const uint32_t hv[4] = {h.x, h.y, h.z, h.w}, lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&hv[j]));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&lv[j]));
    acc = fmaf(a.x + b.x, __uint_as_float(y[2 * j]), acc);
    acc = fmaf(a.y + b.y, __uint_as_float(y[2 * j + 1]), acc);
  }
  return acc;
}

constexpr long long kUmmaSpin = 1ll << 22;      // bounded waits (the MMAs of a stage take about a microsecond):
constexpr unsigned long long kUmmaWaitNs = 200000000ull;   // give up after 2^22 polls or 0.2 s, whichever first

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Wait for the completion of parity `parity` of the mbarrier at shared address bar, bounded.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = globaltimer_ns();
  for (long long n = 0; n < kUmmaSpin; ++n) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((n & 255) == 255 && globaltimer_ns() - t0 > kUmmaWaitNs) return false;
  }
  return false;
}

template <int NCOL>
__global__ void __launch_bounds__(256, 1)
k_colour_umma(const float2* __restrict__ jamps, int64_t nevt, int rows_log2, const int* __restrict__ nrows_dev,
              const uint16_t* __restrict__ cumma, double scale, double* __restrict__ out, int64_t stride,
              const uint8_t* __restrict__ skip, int* __restrict__ err, int stall) {
  using U = Umma<NCOL>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  unsigned char* sB = smem + U::OFF_B;
  float* stg = reinterpret_cast<float*>(smem + U::OFF_STG);
  float* part = reinterpret_cast<float*>(smem + U::OFF_PART);
  int* rexp_all = reinterpret_cast<int*>(smem + U::OFF_EXP);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + U::OFF_BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + U::OFF_BAR + 16);
  int* abort_flag = reinterpret_cast<int*>(smem + U::OFF_BAR + 24);
  uint8_t* vval_all = smem + U::OFF_VAL;                    // [2][VECS]: vector holds a row to compute
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto a_hi = [&](int buf) { return smem + (2 * buf) * U::A_PAD; };
  auto a_lo = [&](int buf) { return smem + (2 * buf + 1) * U::A_PAD; };

  // operands at rest: A's padding chunks stay zero; C in the canonical layout
  for (int i = tid; i < U::OFF_B / 16; i += U::THREADS) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < U::B_BYTES / 16; i += U::THREADS)
    reinterpret_cast<uint4*>(sB)[i] = reinterpret_cast<const uint4*>(cumma)[i];
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_addr(tmem_slot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int nrows = *nrows_dev;
  const int64_t rmask = (int64_t(1) << rows_log2) - 1;
  const int64_t nvec = nevt << rows_log2;                      // vectors in the buffer
  const int64_t nstage = (nvec + U::VECS - 1) / U::VECS;
  const float scale_f = static_cast<float>(scale);
  auto vec_valid = [&](int64_t q) -> bool {
    return q < nvec && (q & rmask) < nrows && (!skip || !skip[q >> rows_log2]);
  };

  float4 pf[U::PF];
  bool pv[U::VPT];
  auto prefetch = [&](int64_t st) {
#pragma unroll
    for (int j = 0; j < U::VPT; ++j) {
      const int v = tid + U::THREADS * j;
      pv[j] = st < nstage && v < U::VECS && vec_valid(st * U::VECS + v);
    }
    const float4* src = reinterpret_cast<const float4*>(jamps) + st * (U::F4);
    const int64_t lim = (nvec - st * U::VECS) * (NCOL * 2 / 4);   // pieces left in the buffer
#pragma unroll
    for (int j = 0; j < U::PF; ++j) {
      const int i = tid + U::THREADS * j;
      pf[j] = (st < nstage && i < U::F4 && i < lim) ? __ldg(src + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };

  // stage st (buffer buf): rows -> A; one thread issues its MMAs
  auto produce = [&](int64_t st, int buf) {
#pragma unroll
    for (int j = 0; j < U::PF; ++j) {
      const int i = tid + U::THREADS * j;
      if (i < U::F4) {
        const int f = 4 * i, v = f / (2 * NCOL), o = f - v * 2 * NCOL;
        float* d = stg + v * U::PITCH + o;
        *reinterpret_cast<float2*>(d) = make_float2(pf[j].x, pf[j].y);
        *reinterpret_cast<float2*>(d + 2) = make_float2(pf[j].z, pf[j].w);
      }
    }
    uint8_t* vval = vval_all + buf * U::VECS;
#pragma unroll
    for (int j = 0; j < U::VPT; ++j)
      if (tid + U::THREADS * j < U::VECS) vval[tid + U::THREADS * j] = pv[j] ? 1 : 0;
    prefetch(st + gridDim.x);
    __syncthreads();
    unsigned char* ahi = a_hi(buf);
    unsigned char* alo = a_lo(buf);
    int* rexp = rexp_all + buf * U::ROWS;
#pragma unroll 1
    for (int pass = 0; pass < U::PASSES; ++pass) {
      const int v = pass * 8 * U::VPL + warp * U::VPL + (lane % U::VPL);
      const int b = lane / U::VPL;
      const bool ok = vval[v] != 0;
      float2 val[U::CPL][8];
      float mre = 0.f, mim = 0.f;
#pragma unroll
      for (int i = 0; i < U::CPL; ++i) {
        const int c = U::VPL == 32 ? i : b + 4 * i;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = 8 * c + j;
          float2 x = make_float2(0.f, 0.f);
          if (ok && c < U::CH && k < NCOL) x = *reinterpret_cast<const float2*>(stg + v * U::PITCH + 2 * k);
          val[i][j] = x;
          mre = fmaxf(mre, fabsf(x.x));
          mim = fmaxf(mim, fabsf(x.y));
        }
      }
      if (U::VPL == 8) {
        mre = fmaxf(mre, __shfl_xor_sync(0xffffffffu, mre, 8));
        mre = fmaxf(mre, __shfl_xor_sync(0xffffffffu, mre, 16));
        mim = fmaxf(mim, __shfl_xor_sync(0xffffffffu, mim, 8));
        mim = fmaxf(mim, __shfl_xor_sync(0xffffffffu, mim, 16));
      }
      int ere = 0, eim = 0;
      if (mre > 0.f) frexpf(mre, &ere);
      if (mim > 0.f) frexpf(mim, &eim);
      const float sre = pow2f_neg(-ere), sim = pow2f_neg(-eim);   // 2^-e (exact for |e| <= 126)
      if (b == 0) {
        rexp[2 * v] = ere;
        rexp[2 * v + 1] = eim;
      }
#pragma unroll
      for (int i = 0; i < U::CPL; ++i) {
        const int c = U::VPL == 32 ? i : b + 4 * i;
        if (c >= U::CH) continue;
        uint32_t hr[4], lr[4], hi_[4], li_[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          split_pair(val[i][2 * j].x * sre, val[i][2 * j + 1].x * sre, hr[j], lr[j]);
          split_pair(val[i][2 * j].y * sim, val[i][2 * j + 1].y * sim, hi_[j], li_[j]);
        }
        const int m = 2 * v;   // real row; the imaginary row m + 1 is 16 bytes further
        const int off = (m & 7) * 16 + (m >> 3) * U::SBO_A + c * 128;
        *reinterpret_cast<uint4*>(ahi + off) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
        *reinterpret_cast<uint4*>(alo + off) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
        *reinterpret_cast<uint4*>(ahi + off + 16) = make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
        *reinterpret_cast<uint4*>(alo + off + 16) = make_uint4(li_[0], li_[1], li_[2], li_[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && !stall) {   // (stall: the diagnostics mode that lets the bounded wait run out)
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t h = smem_addr(ahi), l = smem_addr(alo), bb = smem_addr(sB);
      const uint32_t d = tmem + buf * 128;
#pragma unroll 1
      for (int s = 0; s < U::S; ++s)
#pragma unroll 1
        for (int ks = 0; ks < U::KP / 16; ++ks)
#pragma unroll
          for (int hl = 0; hl < 2; ++hl) {
            const uint32_t a = (hl ? l : h) + s * 16 * U::SBO_A + ks * 256;
            umma_f16(d + s * U::NP, umma_desc(a, 128, U::SBO_A), umma_desc(bb + ks * 256, 128, U::SBO_B), U::IDESC,
                     (ks | hl) != 0);
          }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar + buf))
                   : "memory");
    }
  };

  // stage st (buffer buf), whose MMAs were committed: quadratic forms and outputs
  uint32_t phases = 0;   // bit b: parity of the next completion of buffer b's mbarrier
  auto consume = [&](int64_t st, int buf) -> bool {
    if (!mbar_wait_bounded(smem_addr(bar + buf), (phases >> buf) & 1u)) *abort_flag = 1;
    phases ^= 1u << buf;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (*abort_flag) return false;
    const int64_t q0 = st * U::VECS;
    const unsigned char* ahi = a_hi(buf);
    const unsigned char* alo = a_lo(buf);
    const int* rexp = rexp_all + buf * U::ROWS;
    const uint8_t* vval = vval_all + buf * U::VECS;
    const int qw = warp & 3, hf = warp >> 2;
    const int m = 32 * qw + lane;                          // row within each MMA tile
    const uint32_t taddr = tmem + buf * 128 + (static_cast<uint32_t>(32 * qw) << 16);
    if constexpr (U::S == 1) {
      // one tile: this half's 64 columns = k chunks 8 hf .. 8 hf + 7
      float acc = 0.f;
      const int row_off = (m & 7) * 16 + (m >> 3) * U::SBO_A;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t y[32];
        tmem_ld32(taddr + 64 * hf + 32 * h, y);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int c = 8 * hf + 4 * h + cc;
          if (c < U::CH) {
            const uint4 hv = *reinterpret_cast<const uint4*>(ahi + row_off + c * 128);
            const uint4 lv = *reinterpret_cast<const uint4*>(alo + row_off + c * 128);
            acc = dot8(hv, lv, y + 8 * cc, acc);
          }
        }
      }
      part[hf * 128 + m] = acc;
    } else {
      // this half's S/2 tiles, NP columns each
#pragma unroll
      for (int i = 0; i < U::S / 2; ++i) {
        const int s = hf * (U::S / 2) + i;
        const int mm = 128 * s + m;                        // row of the stage
        const int row_off = (mm & 7) * 16 + (mm >> 3) * U::SBO_A;
        float acc = 0.f;
        if constexpr (U::NP == 16) {
          uint32_t y[16];
          tmem_ld16(taddr + s * U::NP, y);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          acc = dot8(*reinterpret_cast<const uint4*>(ahi + row_off), *reinterpret_cast<const uint4*>(alo + row_off), y, acc);
          if (U::CH > 1)
            acc = dot8(*reinterpret_cast<const uint4*>(ahi + row_off + 128), *reinterpret_cast<const uint4*>(alo + row_off + 128),
                       y + 8, acc);
        } else {
          uint32_t y[32];
          tmem_ld32(taddr + s * U::NP, y);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int c = 0; c < U::CH; ++c)
            acc = dot8(*reinterpret_cast<const uint4*>(ahi + row_off + c * 128),
                       *reinterpret_cast<const uint4*>(alo + row_off + c * 128), y + 8 * c, acc);
        }
        part[s * 128 + m] = acc;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp < 4) {
      const int m2 = 32 * warp + lane;
#pragma unroll
      for (int s = 0; s < U::S; ++s) {
        const float tot = U::S == 1 ? part[m2] + part[128 + m2] : part[s * 128 + m2];
        const int e = rexp[128 * s + m2];
        const float other = __shfl_xor_sync(0xffffffffu, tot, 1);
        const int eo = __shfl_xor_sync(0xffffffffu, e, 1);
        if ((m2 & 1) == 0) {
          const int64_t q = q0 + 64 * s + (m2 >> 1);
          if (vval[64 * s + (m2 >> 1)])
            out[(q & rmask) * stride + (q >> rows_log2)] = combine_rows(tot, 2 * e, other, 2 * eo, scale_f);
        }
      }
    }
    return true;
  };

  int64_t st = blockIdx.x;
  prefetch(st);
  int buf = 0;
  int64_t prev = -1;
  for (;; st += gridDim.x, buf ^= 1) {
    if (st < nstage) produce(st, buf);
    if (prev >= 0) {
      if (!consume(prev, buf ^ 1)) {
        if (tid == 0) atomicCAS(err, 0, static_cast<int>(prev % 1000000) + 1);
        if (st < nstage && !stall)   // the stage just issued: let its MMAs finish (bounded) before the memory goes
          mbar_wait_bounded(smem_addr(bar + buf), (phases >> buf) & 1u);
        break;
      }
    }
    if (st >= nstage) break;
    prev = st;
    __syncthreads();   // the next produce() rewrites the validity flags the combine step above just read
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

// ---- tensor-pipe peak (the f16 MMA denominator of the colour pass's roofline) ----
// Every CTA (one per SM) issues `iters` MMAs of M = 128, N = 256, K = 16 (FP16 operands resident in
// shared memory, FP32 accumulator in tensor memory) from one thread, all into the same accumulator, and
// commits them to one mbarrier.  The operands are small integers (-2..2), so the accumulator is exact:
// CTA 0 writes it out and the host compares it with iters x (A B^T).
constexpr int kPkN = 256;
constexpr uint32_t kPkIdesc = (1u << 4) | (static_cast<uint32_t>(kPkN >> 3) << 17) | (static_cast<uint32_t>(128 >> 4) << 24);

__host__ __device__ inline int pk_a(int r, int k) { return (r * 7 + k * 3) % 5 - 2; }
__host__ __device__ inline int pk_b(int n, int k) { return (n * 5 + k * 11 + 1) % 5 - 2; }

// element (r, k) of an R x 16 K-major operand: 8-row x 16-byte core matrices, the two k halves 128 bytes
// apart, 8-row groups 256 bytes apart (index in halves)
__host__ __device__ inline int pk_off(int r, int k) { return ((r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2) / 2; }

__global__ void __launch_bounds__(128, 1) k_mma_peak(int iters, float* __restrict__ d_out, int* __restrict__ err) {
  __shared__ __align__(128) uint16_t sA[128 * 16];
  __shared__ __align__(128) uint16_t sB[kPkN * 16];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ int timed_out;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < 128 * 16; i += 128)
    sA[pk_off(i >> 4, i & 15)] = __half_as_ushort(__int2half_rn(pk_a(i >> 4, i & 15)));
  for (int i = tid; i < kPkN * 16; i += 128)
    sB[pk_off(i >> 4, i & 15)] = __half_as_ushort(__int2half_rn(pk_b(i >> 4, i & 15)));
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    timed_out = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_addr(&tslot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  if (tid == 0) {
    const uint64_t ad = umma_desc(smem_addr(sA), 128, 256), bd = umma_desc(smem_addr(sB), 128, 256);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) umma_f16(tmem, ad, bd, kPkIdesc, i > 0 ? 1u : 0u);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(&bar))
                 : "memory");
  }
  if (!mbar_wait_bounded(smem_addr(&bar), 0)) timed_out = 1;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (timed_out) {
    if (tid == 0) atomicAdd(err, 1);
  } else if (blockIdx.x == 0) {   // warp w reads tensor-memory lanes 32 w .. 32 w + 31 (rows of D)
    const int row = tid;
#pragma unroll 1
    for (int c = 0; c < kPkN; c += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + (static_cast<uint32_t>(32 * warp) << 16) + c, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 32; ++j) d_out[row * kPkN + c + j] = __uint_as_float(v[j]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

}  // namespace

int colour_tc_cmat_halves(int ncol) {
  switch (ncol) {
    case 2: return TcShape<2>::NP * TcShape<2>::LDH;
    case 6: return TcShape<6>::NP * TcShape<6>::LDH;
    case 24: return TcShape<24>::NP * TcShape<24>::LDH;
    case 120: return TcShape<120>::NP * TcShape<120>::LDH;
    default: return 0;
  }
}

// Host: lay out C (integer numerators) as the padded FP16 operand [NP][LDH] expected by the kernel.
void colour_tc_pack(int ncol, const int64_t* num, uint16_t* out_halves) {
  int LDH = 0;
  switch (ncol) {
    case 2: LDH = TcShape<2>::LDH; break;
    case 6: LDH = TcShape<6>::LDH; break;
    case 24: LDH = TcShape<24>::LDH; break;
    case 120: LDH = TcShape<120>::LDH; break;
    default: return;
  }
  const int total = colour_tc_cmat_halves(ncol);
  for (int i = 0; i < total; ++i) out_halves[i] = 0;
  for (int n = 0; n < ncol; ++n)
    for (int k = 0; k < ncol; ++k) {
      const __half h = __float2half_rn(static_cast<float>(num[static_cast<size_t>(n) * ncol + k]));
      out_halves[n * LDH + k] = __half_as_ushort(h);
    }
}

cudaError_t launch_colour_tc(int ncol, const float2* jamps, int64_t nevt, int rows_alloc, const int* nrows,
                             const void* cmat, double scale, double* out, int64_t stride, cudaStream_t st,
                             const uint8_t* skip) {
  const __half* c = static_cast<const __half*>(cmat);
  switch (ncol) {
    case 2: return launch_tc<2>(jamps, nevt, rows_alloc, nrows, c, scale, out, stride, skip, st);
    case 6: return launch_tc<6>(jamps, nevt, rows_alloc, nrows, c, scale, out, stride, skip, st);
    case 24: return launch_tc<24>(jamps, nevt, rows_alloc, nrows, c, scale, out, stride, skip, st);
    case 120: return launch_tc<120>(jamps, nevt, rows_alloc, nrows, c, scale, out, stride, skip, st);
    default: return cudaErrorInvalidValue;
  }
}


// ---- tensor-memory (tcgen05) colour kernel: host side ----
int colour_umma_halves(int ncol) {
  switch (ncol) {
    case 2: return Umma<2>::B_BYTES / 2;
    case 6: return Umma<6>::B_BYTES / 2;
    case 24: return Umma<24>::B_BYTES / 2;
    case 120: return Umma<120>::B_BYTES / 2;
    default: return 0;
  }
}

// C (integer numerators) as the MMA's B operand: no-swizzle K-major canonical layout, element (n, k) at
// byte (n % 8) 16 + (n / 8) SBO_B + (k / 8) 128 + (k % 8) 2, zero padding up to NP x KP.
void colour_umma_pack(int ncol, const int64_t* num, uint16_t* out_halves) {
  const int total = colour_umma_halves(ncol);
  if (!total) return;
  const int kp = (ncol + 15) / 16 * 16, sbo = kp / 8 * 128;
  for (int i = 0; i < total; ++i) out_halves[i] = 0;
  for (int n = 0; n < ncol; ++n)
    for (int k = 0; k < ncol; ++k) {
      const int byte = (n % 8) * 16 + (n / 8) * sbo + (k / 8) * 128 + (k % 8) * 2;
      out_halves[byte / 2] = __half_as_ushort(__float2half_rn(static_cast<float>(num[static_cast<size_t>(n) * ncol + k])));
    }
}

template <int NCOL>
static cudaError_t launch_umma(const float2* jamps, int64_t nevt, int rows_alloc, const int* nrows, const uint16_t* cumma,
                               double scale, double* out, int64_t stride, const uint8_t* skip, int* err, int stall,
                               cudaStream_t st) {
  using U = Umma<NCOL>;
  int rows_log2 = 0;
  while ((1 << rows_log2) < rows_alloc) ++rows_log2;
  if ((1 << rows_log2) != rows_alloc) return cudaErrorInvalidValue;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  static std::atomic<unsigned long long> configured{0};
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(configured.load(std::memory_order_acquire) & bit)) {
    cudaError_t e = cudaFuncSetAttribute(k_colour_umma<NCOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, U::SMEM);
    if (e != cudaSuccess) return e;
    configured.fetch_or(bit, std::memory_order_release);
  }
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_colour_umma<NCOL>, U::THREADS, U::SMEM) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (per_sm > 2) per_sm = 2;   // 2 x 256 TMEM columns per SM
  const int64_t nstage = ((nevt << rows_log2) + U::VECS - 1) / U::VECS;
  int64_t blocks = static_cast<int64_t>(nsm) * per_sm;
  if (blocks > nstage) blocks = nstage;
  if (blocks < 1) return cudaSuccess;
  { k_colour_umma<NCOL><<<static_cast<unsigned>(blocks), U::THREADS, U::SMEM, st>>>(jamps, nevt, rows_log2, nrows, cumma, scale,
                                                                                  out, stride, skip, err, stall); mg::note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_colour_umma(int ncol, const float2* jamps, int64_t nevt, int rows_alloc, const int* nrows,
                               const void* cumma, double scale, double* out, int64_t stride, cudaStream_t st,
                               const uint8_t* skip, int* err, int stall) {
  const uint16_t* c = static_cast<const uint16_t*>(cumma);
  switch (ncol) {
    case 2: return launch_umma<2>(jamps, nevt, rows_alloc, nrows, c, scale, out, stride, skip, err, stall, st);
    case 6: return launch_umma<6>(jamps, nevt, rows_alloc, nrows, c, scale, out, stride, skip, err, stall, st);
    case 24: return launch_umma<24>(jamps, nevt, rows_alloc, nrows, c, scale, out, stride, skip, err, stall, st);
    case 120: return launch_umma<120>(jamps, nevt, rows_alloc, nrows, c, scale, out, stride, skip, err, stall, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mg

extern "C" mg_status mg_measure_mma_peak(int iters, double* flops_per_s) {
  if (!flops_per_s || iters < 1 || iters > (1 << 16)) return MG_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return MG_ECUDA;
  }
  float* out = nullptr;
  int* err = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mg_status rc = MG_OK;
  if (mg::dev_alloc(&out, sizeof(float) * 128 * mg::kPkN) != cudaSuccess || mg::dev_alloc(&err, sizeof(int)) != cudaSuccess) {
    rc = MG_ENOMEM;
  } else if (cudaMemset(err, 0, sizeof(int)) != cudaSuccess ||
             cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = MG_ECUDA;
  } else {
    { mg::k_mma_peak<<<nsm, 128, 0, st>>>(iters / 8 + 1, out, err); mg::note_launch(); }   // warm-up
    cudaEventRecord(e0, st);
    { mg::k_mma_peak<<<nsm, 128, 0, st>>>(iters, out, err); mg::note_launch(); }
    cudaEventRecord(e1, st);
    std::vector<float> d(128 * mg::kPkN);
    int nerr = 0;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaMemcpy(d.data(), out, d.size() * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&nerr, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = MG_ECUDA;
    } else if (nerr) {
      rc = MG_ETIMEOUT;
    } else {
      for (int r = 0; r < 128 && rc == MG_OK; ++r)
        for (int n = 0; n < mg::kPkN; ++n) {
          int dot = 0;
          for (int k = 0; k < 16; ++k) dot += mg::pk_a(r, k) * mg::pk_b(n, k);
          if (d[r * mg::kPkN + n] != static_cast<float>(static_cast<int64_t>(dot) * iters)) { rc = MG_ECUDA; break; }
        }
      if (rc == MG_OK) *flops_per_s = 2.0 * 128 * mg::kPkN * 16 * static_cast<double>(iters) * nsm / (ms * 1e-3);
    }
  }
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  mg::dev_free(out);
  mg::dev_free(err);
  return rc;
}
