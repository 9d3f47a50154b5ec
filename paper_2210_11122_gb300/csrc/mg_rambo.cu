// mg_rambo.cu -- random numbers -> momenta on the device (the paper's standalone workflow,
// Sec. 1 / Fig. 1: a simplified random-number generator and phase-space sampler executed fully
// on the GPU, feeding the matrix-element kernel).
//
//  * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the 4x32 S-box with
//    multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 / 0xBB67AE85.
//    Event e, final-state particle j: counter {e_lo, e_hi, j, 0}, key {seed_lo, seed_hi};
//    uniforms u = (x + 0.5) 2^-32 (exact in FP64, strictly inside (0,1)).
//  * RAMBO (Kleiss, Stirling, Ellis, Comput. Phys. Commun. 40 (1986) 359): isotropic massless
//    q_i with energy density q0 exp(-q0), conformal map onto (sqrt s, 0, 0, 0), then the massive
//    rescaling k_i = (sqrt(m_i^2 + xi^2 |p_i|^2), xi p_i) with xi from Newton's method.
// One thread per event; the momenta are written in the AoSoA layout of mg.h (page of 32 events,
// so every store of a warp is one 256-byte line).
#include <cuda_runtime.h>

#include "mg_internal.h"

namespace mg {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__global__ void k_philox(uint64_t seed, int64_t nevt, int nfinal, uint32_t* __restrict__ words) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= nevt * nfinal) return;
  const int64_t e = t / nfinal;
  const uint32_t j = static_cast<uint32_t>(t - e * nfinal);
  const uint4 x = philox4x32_10(make_uint4(static_cast<uint32_t>(e), static_cast<uint32_t>(e >> 32), j, 0u),
                                make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)));
  reinterpret_cast<uint4*>(words)[t] = x;
}

__device__ __forceinline__ double unif(uint32_t x) { return (static_cast<double>(x) + 0.5) * 0x1p-32; }

// NF final-state particles: t, tbar (mass mt) and NF-2 massless gluons.
template <int NF>
__global__ void __launch_bounds__(128) k_rambo(uint64_t seed, int64_t e0, int64_t nevt, double sqrts, double mt,
                                               double w0, double* __restrict__ mom, double* __restrict__ wgt,
                                               unsigned long long* __restrict__ nbad) {
  const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;   // output position
  if (e >= nevt) return;
  const int64_t ev = e0 + e;                                                         // Philox event counter
  constexpr int npar = NF + 2;
  const uint2 key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  double q[NF][4];
  double Q0 = 0, Q1 = 0, Q2 = 0, Q3 = 0;
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const uint4 x = philox4x32_10(
        make_uint4(static_cast<uint32_t>(ev), static_cast<uint32_t>(ev >> 32), static_cast<uint32_t>(j), 0u), key);
    const double u0 = unif(x.x), u1 = unif(x.y), u2 = unif(x.z), u3 = unif(x.w);
    const double c = 2.0 * u0 - 1.0;
    const double s = 2.0 * sqrt(u0 * (1.0 - u0));   // sqrt(1 - c^2)
    double sn, cs;
    sincospi(2.0 * u1, &sn, &cs);
    const double q0 = -log(u2 * u3);
    q[j][0] = q0;
    q[j][1] = q0 * s * cs;
    q[j][2] = q0 * s * sn;
    q[j][3] = q0 * c;
    Q0 += q[j][0]; Q1 += q[j][1]; Q2 += q[j][2]; Q3 += q[j][3];
  }
  const double M = sqrt(Q0 * Q0 - Q1 * Q1 - Q2 * Q2 - Q3 * Q3);
  const double b1 = -Q1 / M, b2 = -Q2 / M, b3 = -Q3 / M;
  const double gam = Q0 / M, a = 1.0 / (1.0 + gam), x = sqrts / M;
  double p[NF][4];
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    const double bq = b1 * q[j][1] + b2 * q[j][2] + b3 * q[j][3];
    p[j][0] = x * (gam * q[j][0] + bq);
    p[j][1] = x * (q[j][1] + b1 * q[j][0] + a * bq * b1);
    p[j][2] = x * (q[j][2] + b2 * q[j][0] + a * bq * b2);
    p[j][3] = x * (q[j][3] + b3 * q[j][0] + a * bq * b3);
  }
  double w = w0;
  if (mt > 0.0) {
    const double msum = 2.0 * mt;
    double xi = sqrt(1.0 - (msum / sqrts) * (msum / sqrts));
    bool ok = false;
    for (int it = 0; it < 50; ++it) {
      double f = -sqrts, fp = 0.0;
#pragma unroll
      for (int j = 0; j < NF; ++j) {
        const double m = j < 2 ? mt : 0.0;
        const double ej = sqrt(m * m + xi * xi * p[j][0] * p[j][0]);
        f += ej;
        fp += xi * p[j][0] * p[j][0] / ej;
      }
      if (fabs(f) <= 1e-14 * sqrts) { ok = true; break; }
      xi -= f / fp;
    }
    if (!ok) atomicAdd(nbad, 1ull);
    double prod = 1.0, sumv = 0.0;
#pragma unroll
    for (int j = 0; j < NF; ++j) {
      const double m = j < 2 ? mt : 0.0;
      const double ej = sqrt(m * m + xi * xi * p[j][0] * p[j][0]);
      const double v = xi * p[j][0];
      p[j][1] *= xi; p[j][2] *= xi; p[j][3] *= xi;
      p[j][0] = ej;
      prod *= v / ej;
      sumv += v * v / ej;
    }
    double xp = 1.0;
#pragma unroll
    for (int i = 0; i < 2 * NF - 3; ++i) xp *= xi;
    w *= xp * prod * sqrts / sumv;
  }
  // AoSoA store: page = e / 32, lane = e % 32
  const int64_t page = e / kPage;
  const int lane = static_cast<int>(e % kPage);
  double* base = mom + page * npar * 4 * kPage + lane;
  const double h = 0.5 * sqrts;
  const double beams[2][4] = {{h, 0.0, 0.0, h}, {h, 0.0, 0.0, -h}};
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) base[(i * 4 + mu) * kPage] = beams[i][mu];
#pragma unroll
  for (int j = 0; j < NF; ++j)
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) base[((j + 2) * 4 + mu) * kPage] = p[j][mu];
  if (wgt) wgt[e] = w;
}

cudaError_t launch_philox(uint64_t seed, int64_t nevt, int nfinal, uint32_t* words, cudaStream_t st) {
  const int64_t n = nevt * nfinal;
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  if (blocks > 0) { k_philox<<<static_cast<unsigned>(blocks), threads, 0, st>>>(seed, nevt, nfinal, words); mg::note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_rambo(int K, uint64_t seed, int64_t e0, int64_t nevt, double sqrts, double mt, double w0,
                         double* mom, double* wgt, unsigned long long* nbad, cudaStream_t st) {
  const int threads = 128;
  const unsigned blocks = static_cast<unsigned>((nevt + threads - 1) / threads);
  if (blocks == 0) return cudaSuccess;
  switch (K) {
    case 2: { k_rambo<2><<<blocks, threads, 0, st>>>(seed, e0, nevt, sqrts, mt, w0, mom, wgt, nbad); mg::note_launch(); } break;
    case 3: { k_rambo<3><<<blocks, threads, 0, st>>>(seed, e0, nevt, sqrts, mt, w0, mom, wgt, nbad); mg::note_launch(); } break;
    case 4: { k_rambo<4><<<blocks, threads, 0, st>>>(seed, e0, nevt, sqrts, mt, w0, mom, wgt, nbad); mg::note_launch(); } break;
    case 5: { k_rambo<5><<<blocks, threads, 0, st>>>(seed, e0, nevt, sqrts, mt, w0, mom, wgt, nbad); mg::note_launch(); } break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mg
