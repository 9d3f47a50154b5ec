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

#include <cuda_fp16.h>
#include <cuda_runtime.h>

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

}  // namespace mg
