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
//     a . Y is formed in FP32 with the unsplit (FP32) a, then unscaled exactly.
// Relative error per (event, helicity) ~1e-7 (the colour matrices are well conditioned: kappa <= 16).
// Rows: jamps[(e * rows_alloc + r) * ncol + sigma] (FP32 complex), r < *nrows_dev; output:
// out[r * stride + e] = colour sum * scale, in FP64.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "mg_internal.h"
#include "mg_kernels.h"

namespace mg {
namespace {

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
  static constexpr int NT = (NCOL + 7) / 8;          // output column tiles of 8
  static constexpr int NP = NT * 8;
  static constexpr int LDH = KP + 8;                 // half pitch (breaks bank conflicts)
  static constexpr int LDF = KP + 4;                 // float pitch
  static constexpr int WARPS = 4;
  static constexpr size_t smem_bytes() {
    return sizeof(__half) * (size_t(NP) * LDH + size_t(WARPS) * 2 * 16 * LDH) + sizeof(float) * size_t(WARPS) * 16 * LDF;
  }
};

template <int NCOL>
__global__ void __launch_bounds__(128) k_colour_tc(const float2* __restrict__ jamps, int64_t nevt, int rows_alloc,
                                                   const int* __restrict__ nrows_dev, const __half* __restrict__ cmat,
                                                   double scale, double* __restrict__ out, int64_t stride,
                                                   const uint8_t* __restrict__ skip) {
  using S = TcShape<NCOL>;
  constexpr int KP = S::KP, NT = S::NT, NP = S::NP, LDH = S::LDH, LDF = S::LDF;
  extern __shared__ __align__(16) unsigned char smem[];
  __half* sC = reinterpret_cast<__half*>(smem);                       // [NP][LDH]: C[n][k]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __half* sHi = sC + NP * LDH + warp * 2 * 16 * LDH;                  // [16][LDH]
  __half* sLo = sHi + 16 * LDH;
  float* sF = reinterpret_cast<float*>(sC + NP * LDH + S::WARPS * 2 * 16 * LDH) + warp * 16 * LDF;   // [16][LDF]

  for (int i = threadIdx.x; i < NP * LDH; i += blockDim.x) sC[i] = cmat[i];
  __syncthreads();

  const int nrows = *nrows_dev;
  const int64_t npairs = nevt * nrows;
  const int g = lane >> 2, q = lane & 3;
  for (int64_t tile = static_cast<int64_t>(blockIdx.x) * S::WARPS + warp; tile * 8 < npairs;
       tile += static_cast<int64_t>(gridDim.x) * S::WARPS) {
    // stage 8 (event, helicity) jamp vectors as 16 rows: row 2p = Re, 2p+1 = Im of pair p
    for (int idx = lane; idx < 8 * KP; idx += 32) {
      const int p = idx / KP, b = idx - p * KP;
      const int64_t qq = tile * 8 + p;
      float2 v = make_float2(0.f, 0.f);
      if (qq < npairs && b < NCOL) {
        const int64_t e = qq / nrows;
        const int r = static_cast<int>(qq - e * nrows);
        if (!skip || !skip[e]) v = jamps[(e * rows_alloc + r) * NCOL + b];   // skipped events: no jamps
      }
      sF[(2 * p) * LDF + b] = v.x;
      sF[(2 * p + 1) * LDF + b] = v.y;
    }
    __syncwarp();
    // per-row power-of-two scale and hi/lo split: two lanes per row
    const int row = lane >> 1, half = lane & 1;
    float mx = 0.f;
    for (int b = half; b < KP; b += 2) mx = fmaxf(mx, fabsf(sF[row * LDF + b]));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    int ex = 0;
    if (mx > 0.f) frexpf(mx, &ex);
    const float sc = ldexpf(1.f, -ex);
    for (int b = half; b < KP; b += 2) {
      const float t = sF[row * LDF + b] * sc;
      const __half hi = __float2half_rn(t);
      const __half lo = __float2half_rn((t - __half2float(hi)) * 2048.f);
      sF[row * LDF + b] = t;
      sHi[row * LDH + b] = hi;
      sLo[row * LDH + b] = lo;
    }
    __syncwarp();
    // Y = C a (rows g and g+8 of this thread's fragments), then the quadratic form a . Y
    float s0 = 0.f, s1 = 0.f;
#pragma unroll 1
    for (int nt = 0; nt < NT; ++nt) {
      float dh[4] = {0.f, 0.f, 0.f, 0.f}, dl[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < KP / 16; ++ks) {
        const int k0 = ks * 16 + q * 2;
        uint32_t ah[4], al[4], bf[2];
        ah[0] = *reinterpret_cast<const uint32_t*>(sHi + g * LDH + k0);
        ah[1] = *reinterpret_cast<const uint32_t*>(sHi + (g + 8) * LDH + k0);
        ah[2] = *reinterpret_cast<const uint32_t*>(sHi + g * LDH + k0 + 8);
        ah[3] = *reinterpret_cast<const uint32_t*>(sHi + (g + 8) * LDH + k0 + 8);
        al[0] = *reinterpret_cast<const uint32_t*>(sLo + g * LDH + k0);
        al[1] = *reinterpret_cast<const uint32_t*>(sLo + (g + 8) * LDH + k0);
        al[2] = *reinterpret_cast<const uint32_t*>(sLo + g * LDH + k0 + 8);
        al[3] = *reinterpret_cast<const uint32_t*>(sLo + (g + 8) * LDH + k0 + 8);
        const int n = nt * 8 + g;
        bf[0] = *reinterpret_cast<const uint32_t*>(sC + n * LDH + k0);
        bf[1] = *reinterpret_cast<const uint32_t*>(sC + n * LDH + k0 + 8);
        mma16816(dh, ah, bf);
        mma16816(dl, al, bf);
      }
      const int c = nt * 8 + q * 2;
      const float r = 1.f / 2048.f;
      s0 = fmaf(sF[g * LDF + c], fmaf(dl[0], r, dh[0]), s0);
      s0 = fmaf(sF[g * LDF + c + 1], fmaf(dl[1], r, dh[1]), s0);
      s1 = fmaf(sF[(g + 8) * LDF + c], fmaf(dl[2], r, dh[2]), s1);
      s1 = fmaf(sF[(g + 8) * LDF + c + 1], fmaf(dl[3], r, dh[3]), s1);
    }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    // undo the row scales (exact powers of two): rows g and g+8 belong to lanes 2g and 2(g+8)
    const float sc0 = __shfl_sync(0xffffffffu, sc, 2 * g);
    const float sc1 = __shfl_sync(0xffffffffu, sc, 2 * (g + 8));
    const double v0 = static_cast<double>(s0) / (static_cast<double>(sc0) * sc0);
    const double v1 = static_cast<double>(s1) / (static_cast<double>(sc1) * sc1);
    // rows 2p (Re) and 2p+1 (Im) of a pair sit in quads g and g^1
    const double w0 = v0 + __shfl_xor_sync(0xffffffffu, v0, 4);
    const double w1 = v1 + __shfl_xor_sync(0xffffffffu, v1, 4);
    if (q == 0 && (g & 1) == 0) {
      const int64_t qa = tile * 8 + g / 2, qb = tile * 8 + 4 + g / 2;
      if (qa < npairs) {
        const int64_t e = qa / nrows;
        if (!skip || !skip[e]) out[(qa - e * nrows) * stride + e] = w0 * scale;
      }
      if (qb < npairs) {
        const int64_t e = qb / nrows;
        if (!skip || !skip[e]) out[(qb - e * nrows) * stride + e] = w1 * scale;
      }
    }
    __syncwarp();
  }
}

template <int NCOL>
cudaError_t launch_tc(const float2* jamps, int64_t nevt, int rows_alloc, const int* nrows, const __half* cmat,
                      double scale, double* out, int64_t stride, const uint8_t* skip, cudaStream_t st) {
  using S = TcShape<NCOL>;
  const size_t smem = S::smem_bytes();
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_colour_tc<NCOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (nevt * rows_alloc + 7) / 8;
  int64_t blocks = (tiles + S::WARPS - 1) / S::WARPS;
  const int64_t cap = static_cast<int64_t>(nsm) * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) return cudaSuccess;
  k_colour_tc<NCOL><<<static_cast<unsigned>(blocks), 128, smem, st>>>(jamps, nevt, rows_alloc, nrows, cmat, scale, out,
                                                                       stride, skip);
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
