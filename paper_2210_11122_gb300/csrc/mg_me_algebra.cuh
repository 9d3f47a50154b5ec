// mg_me_algebra.cuh -- device algebra shared by the matrix-element kernels (mg_me2.cu, mg_me3.cu):
// complex FMA chains, HELAS-convention external wavefunctions (helicity spinors of the tops in the
// chiral basis, transverse gluon polarisations), the Feynman-gauge three- and four-gluon vertices
// and the quark-line vertex/propagator contracted with currents, the colour quadratic form, and the
// per-event record (subset momenta, propagator factors, wavefunctions) that a per-event kernel
// computes once in FP64 for every helicity of the event.
#pragma once

#include <cuda_runtime.h>

#include "mg_internal.h"
#include "mg_kernels.h"

namespace mg {
namespace dd {

// Double-float number: an unevaluated sum hi + lo of two FP32 values, |lo| <= ulp(hi) / 2, carrying
// ~48 significant bits with FP32 instructions only (Dekker, Numer. Math. 18 (1971) 224; Knuth, TAOCP
// vol. 2, 4.2.2: error-free sum of two floats; the product error from one FMA).  Every step uses the
// non-contractible __fadd_rn / __fmul_rn intrinsics so that the compiler cannot fuse an error-free
// transformation into an FMA.  Sums use the short form (no renormalisation of the low parts first),
// whose relative error is ~2^-46 times the cancellation ratio |a| / |a + b|.
struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __device__ df(double x) : hi(static_cast<float>(x)), lo(static_cast<float>(x - static_cast<double>(static_cast<float>(x)))) {}
  __device__ explicit operator double() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df operator+(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df fma(df a, df b, df c) {   // a b + c
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const df s = two_sum(p, c.hi);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

}  // namespace dd
}  // namespace mg

namespace mg {
namespace v2 {

template <class T>
struct cx {
  T r, i;
};

template <class T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {fma(a.r, b.r, -(a.i * b.i)), fma(a.r, b.i, a.i * b.r)};
}
template <class T> __device__ __forceinline__ void cmac(cx<T>& c, cx<T> a, cx<T> b) {   // c += a b
  c.r = fma(a.r, b.r, c.r); c.r = fma(-a.i, b.i, c.r);
  c.i = fma(a.r, b.i, c.i); c.i = fma(a.i, b.r, c.i);
}
template <class T> __device__ __forceinline__ void cmsub(cx<T>& c, cx<T> a, cx<T> b) {  // c -= a b
  c.r = fma(-a.r, b.r, c.r); c.r = fma(a.i, b.i, c.r);
  c.i = fma(-a.r, b.i, c.i); c.i = fma(-a.i, b.r, c.i);
}
template <class T> __device__ __forceinline__ void cmacr(cx<T>& c, T s, cx<T> a) {      // c += s a, s real
  c.r = fma(s, a.r, c.r); c.i = fma(s, a.i, c.i);
}
template <class T> __device__ __forceinline__ cx<T> cscale(T s, cx<T> a) { return {s * a.r, s * a.i}; }
template <class T> __device__ __forceinline__ cx<T> cneg(cx<T> a) { return {-a.r, -a.i}; }

// Minkowski dot products
template <class T> __device__ __forceinline__ cx<T> mdot(const cx<T>* a, const cx<T>* b) {
  cx<T> r = cmul(a[0], b[0]);
  cmsub(r, a[1], b[1]); cmsub(r, a[2], b[2]); cmsub(r, a[3], b[3]);
  return r;
}
template <class T> __device__ __forceinline__ cx<T> mdotr(const cx<T>* a, const T* p) {
  cx<T> r = cscale(p[0], a[0]);
  cmacr(r, -p[1], a[1]); cmacr(r, -p[2], a[2]); cmacr(r, -p[3], a[3]);
  return r;
}

template <int K> struct Sizes;
template <> struct Sizes<2> { static constexpr int ncol = 2, nseq = 2, nfull = 1; };
template <> struct Sizes<3> { static constexpr int ncol = 6, nseq = 6, nfull = 3; };
template <> struct Sizes<4> { static constexpr int ncol = 24, nseq = 22, nfull = 12; };
template <> struct Sizes<5> { static constexpr int ncol = 120, nseq = 105, nfull = 60; };

__device__ __forceinline__ int rslot(int16_t r) { return r >> 1; }
__device__ __forceinline__ bool rneg(int16_t r) { return r & 1; }

// ---- FP64 helpers of the per-event record ----
// Reciprocal and reciprocal square root for the FP32-amplitude path's record: an FP32 seed refined by
// one Newton-Raphson step in FP64 (r <- r (2 - x r) for 1/x, y <- y (3 - x y^2) / 2 for 1/sqrt(x); each
// step squares the seed's relative error, ~2^-23 -> ~2^-45), so that the values stored in FP32 carry
// only their final rounding, at a fraction of the FP64 cost of a correctly rounded division.  Outside
// 2^-99 < |x| < 2^99 (tested on the exponent bits, on the integer pipe) the FP64 operation is used.
__device__ __forceinline__ bool in_f32_range(double x) {
  const int e = (__double2hiint(x) >> 20) & 0x7ff;
  return e > 1023 - 99 && e < 1023 + 99;
}
__device__ __forceinline__ double rcp_nr(double x) {
  if (!in_f32_range(x)) return 1.0 / x;
  const double r0 = static_cast<double>(__frcp_rn(static_cast<float>(x)));
  return r0 * fma(-x, r0, 2.0);
}
__device__ __forceinline__ double rsqrt_nr(double x) {
  if (!(__double2hiint(x) > 0 && in_f32_range(x))) return rsqrt(x);
  const double y0 = static_cast<double>(rsqrtf(static_cast<float>(x)));
  return y0 * fma(-0.5 * x * y0, y0, 1.5);
}
// NR = false: correctly rounded FP64 operations (FP64 path); true: the Newton-refined forms above
template <bool NR> __device__ __forceinline__ double r_sqrt(double x) {
  if constexpr (NR) return x > 0.0 ? x * rsqrt_nr(x) : 0.0;
  else return sqrt(x);
}
template <bool NR> __device__ __forceinline__ double r_rsqrt(double x) {
  if constexpr (NR) return rsqrt_nr(x);
  else return rsqrt(x);
}
template <bool NR> __device__ __forceinline__ double r_div(double a, double b) {
  if constexpr (NR) return a * rcp_nr(b);
  else return a / b;
}

// ---- external wavefunctions (FP64 arithmetic) ----
// two-component helicity eigenstates chi_lam of the direction of p
template <bool NR>
__device__ __forceinline__ void chi2(const double* p, double pa, int lam, cx<double>* c) {
  const double px = p[1], py = p[2], pz = p[3];
  const double pt2 = px * px + py * py;
  const double apz = pz >= 0.0 ? pa + pz : r_div<NR>(pt2, pa - pz);
  if (apz > 0.0) {
    const double n = r_rsqrt<NR>(2.0 * pa * apz);
    if (lam > 0) { c[0] = {apz * n, 0.0}; c[1] = {px * n, py * n}; }
    else { c[0] = {-px * n, py * n}; c[1] = {apz * n, 0.0}; }
  } else {
    if (lam > 0) { c[0] = {0.0, 0.0}; c[1] = {1.0, 0.0}; }
    else { c[0] = {-1.0, 0.0}; c[1] = {0.0, 0.0}; }
  }
}

// |p|, sqrt(E + |p|) and m / sqrt(E + |p|) of a massive fermion
template <bool NR>
__device__ __forceinline__ void spinor_norms(const double* p, double m, double& pa, double& sp, double& sm) {
  pa = r_sqrt<NR>(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  if constexpr (NR) {
    const double rs = rsqrt_nr(p[0] + pa);
    sp = (p[0] + pa) * rs;
    sm = m > 0.0 ? m * rs : 0.0;
  } else {
    sp = sqrt(p[0] + pa);
    sm = m > 0.0 ? m / sp : 0.0;
  }
}

template <class T>
__device__ __forceinline__ void top_ubar(const double* p, double m, int lam, cx<T>* w) {
  constexpr bool NR = sizeof(T) == 4;
  double pa, sp, sm;
  spinor_norms<NR>(p, m, pa, sp, sm);
  cx<double> c[2];
  chi2<NR>(p, pa, lam, c);
  const double fl = lam > 0 ? sm : sp, fr = lam > 0 ? sp : sm;
  w[0] = {T(fr * c[0].r), T(-fr * c[0].i)}; w[1] = {T(fr * c[1].r), T(-fr * c[1].i)};
  w[2] = {T(fl * c[0].r), T(-fl * c[0].i)}; w[3] = {T(fl * c[1].r), T(-fl * c[1].i)};
}

template <class T>
__device__ __forceinline__ void top_v(const double* p, double m, int lam, cx<T>* w) {
  constexpr bool NR = sizeof(T) == 4;
  double pa, sp, sm;
  spinor_norms<NR>(p, m, pa, sp, sm);
  cx<double> c[2];
  chi2<NR>(p, pa, -lam, c);
  const double fl = lam > 0 ? -sp : sm, fr = lam > 0 ? sm : -sp;
  w[0] = {T(fl * c[0].r), T(fl * c[0].i)}; w[1] = {T(fl * c[1].r), T(fl * c[1].i)};
  w[2] = {T(fr * c[0].r), T(fr * c[0].i)}; w[3] = {T(fr * c[1].r), T(fr * c[1].i)};
}

// Transverse polarisation basis of a gluon of momentum k, pre-scaled by 1/sqrt(2):
// pol = (e_theta / sqrt2 [3 components], e_phi / sqrt2 [x, y]; e_phi has no z component).  Correctly
// rounded FP64 on the FP64 path; Newton-refined reciprocals on the FP32-amplitude path.
template <class T>
__device__ __forceinline__ void gluon_pol(const double* k, T* pol) {
  const double kx = k[1], ky = k[2], kz = k[3];
  const double kt2 = kx * kx + ky * ky;
  const double r = 0.70710678118654752440;
  double et[3], ep[2];
  if (kt2 > 0.0) {
    if constexpr (sizeof(T) == 8) {
      const double kt = sqrt(kt2), ka = sqrt(kt2 + kz * kz);
      const double inv = 1.0 / (ka * kt);
      et[0] = kx * kz * inv; et[1] = ky * kz * inv; et[2] = -kt / ka;
      ep[0] = -ky / kt; ep[1] = kx / kt;
    } else {
      const double rt = rsqrt_nr(kt2), ra = rsqrt_nr(kt2 + kz * kz);
      const double inv = ra * rt;
      et[0] = kx * kz * inv; et[1] = ky * kz * inv; et[2] = -(kt2 * rt) * ra;
      ep[0] = -ky * rt; ep[1] = kx * rt;
    }
  } else {
    et[0] = kz < 0.0 ? -1.0 : 1.0; et[1] = 0.0; et[2] = 0.0;
    ep[0] = 0.0; ep[1] = 1.0;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) pol[i] = T(r * et[i]);
  pol[3] = T(r * ep[0]);
  pol[4] = T(r * ep[1]);
}

// External gluon current of helicity lam: eps = (-lam e_theta + i s e_phi) / sqrt2, s = +1 for an
// outgoing gluon (eps*), -1 for an incoming one; from the pre-scaled basis by exact sign flips.
template <class T>
__device__ __forceinline__ void ext_gluon(const T* pol, int lam, bool outgoing, cx<T>* w) {
  w[0] = {T(0), T(0)};
  w[1] = {lam > 0 ? -pol[0] : pol[0], outgoing ? pol[3] : -pol[3]};
  w[2] = {lam > 0 ? -pol[1] : pol[1], outgoing ? pol[4] : -pol[4]};
  w[3] = {lam > 0 ? -pol[2] : pol[2], T(0)};
}

// ---- current algebra ----
// acc += s * V3(JL, JR) with incoming momenta PL, PR.  The Feynman-gauge vertex contracted with the
// two currents is (JL.JR)(PL - PR) + (JL.(PL + 2 PR)) JR - (JR.(2 PL + PR)) JL; Berends-Giele
// currents of on-shell transverse gluons are conserved (P.J(P) = 0 exactly), so the JL.PL and JR.PR
// parts vanish and the vertex is evaluated as (JL.JR)(PL - PR) + 2 (JL.PR) JR - 2 (JR.PL) JL: the
// same value, without adding the rounding noise of two vanishing products (which 1/P^2 factors of
// nearly collinear pairs amplify in FP32).
template <class T>
__device__ __forceinline__ void v3_acc(cx<T>* acc, const cx<T>* JL, const cx<T>* JR, const T* PL, const T* PR, bool neg) {
  T d[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) d[m] = PL[m] - PR[m];
  cx<T> jj = mdot(JL, JR), cl = mdotr(JL, PR), cr = mdotr(JR, PL);
  const T two = neg ? T(-2) : T(2);
  if (neg) jj = cneg(jj);
  cl = cscale(two, cl);
  cr = cscale(two, cr);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    cmacr(acc[m], d[m], jj);
    cmac(acc[m], cl, JR[m]);
    cmsub(acc[m], cr, JL[m]);
  }
}

// acc += s * g * V4(JA, JB, JC), V4 = (JA.JB) JC + (JB.JC) JA - 2 (JA.JC) JB
template <class T>
__device__ __forceinline__ void v4_acc(cx<T>* acc, const cx<T>* JA, const cx<T>* JB, const cx<T>* JC, T g, bool neg) {
  const T s = neg ? -g : g;
  const cx<T> ab = cscale(s, mdot(JA, JB)), bc = cscale(s, mdot(JB, JC)), ac = cscale(T(2) * s, mdot(JA, JC));
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    cmac(acc[m], ab, JC[m]);
    cmac(acc[m], bc, JA[m]);
    cmsub(acc[m], ac, JB[m]);
  }
}

// gamma.J in the chiral basis by its four distinct entries (sign (+/-) applied), so that several row
// spinors can be multiplied into the same current
template <class T> struct Slash { cx<T> a, b, jm, jp; };
template <class T>
__device__ __forceinline__ Slash<T> slash_of(const cx<T>* J, bool neg) {
  Slash<T> g;
  g.jm = {J[1].r + J[2].i, J[1].i - J[2].r};   // J1 - i J2
  g.jp = {J[1].r - J[2].i, J[1].i + J[2].r};   // J1 + i J2
  g.a = {J[0].r + J[3].r, J[0].i + J[3].i};
  g.b = {J[0].r - J[3].r, J[0].i - J[3].i};
  if (neg) { g.jm = cneg(g.jm); g.jp = cneg(g.jp); g.a = cneg(g.a); g.b = cneg(g.b); }
  return g;
}

// acc += s g  (row spinor s times a current's gamma.J entries)
template <class T>
__device__ __forceinline__ void row_slash_acc(cx<T>* acc, const cx<T>* s, const Slash<T>& g) {
  cmac(acc[0], s[2], g.a); cmac(acc[0], s[3], g.jp);
  cmac(acc[1], s[2], g.jm); cmac(acc[1], s[3], g.b);
  cmac(acc[2], s[0], g.b); cmsub(acc[2], s[1], g.jp);
  cmac(acc[3], s[1], g.a); cmsub(acc[3], s[0], g.jm);
}

// acc (+/-)= s gamma.J  (row spinor s, gluon current J)
template <class T>
__device__ __forceinline__ void row_gamma_acc(cx<T>* acc, const cx<T>* s, const cx<T>* J, bool neg) {
  row_slash_acc(acc, s, slash_of(J, neg));
}

// (gamma.J) v
template <class T>
__device__ __forceinline__ void gamma_col(const cx<T>* J, const cx<T>* v, cx<T>* o) {
  const cx<T> jm = {J[1].r + J[2].i, J[1].i - J[2].r};
  const cx<T> jp = {J[1].r - J[2].i, J[1].i + J[2].r};
  const cx<T> a = {J[0].r + J[3].r, J[0].i + J[3].i}, b = {J[0].r - J[3].r, J[0].i - J[3].i};
  o[0] = cmul(b, v[2]); cmsub(o[0], jm, v[3]);
  o[1] = cmul(a, v[3]); cmsub(o[1], jp, v[2]);
  o[2] = cmul(a, v[0]); cmac(o[2], jm, v[1]);
  o[3] = cmul(jp, v[0]); cmac(o[3], b, v[1]);
}

// quark propagator with factor: o = s (Qslash + m) f, coefficients q = {(Q0+Q3) f, (Q0-Q3) f, Q1 f, Q2 f, m f}
template <class T>
__device__ __forceinline__ void row_prop(const cx<T>* s, const T* q, cx<T>* o) {
  const T qa = q[0], qb = q[1], q1 = q[2], q2 = q[3], qm = q[4];
  // o0 = qa s2 + (q1 + i q2) s3 + qm s0 ; o1 = (q1 - i q2) s2 + qb s3 + qm s1
  // o2 = qb s0 - (q1 + i q2) s1 + qm s2 ; o3 = qa s1 - (q1 - i q2) s0 + qm s3
  const cx<T> qp = {q1, q2}, qn = {q1, -q2};
  o[0] = cscale(qa, s[2]); cmac(o[0], qp, s[3]); cmacr(o[0], qm, s[0]);
  o[1] = cscale(qb, s[3]); cmac(o[1], qn, s[2]); cmacr(o[1], qm, s[1]);
  o[2] = cscale(qb, s[0]); cmsub(o[2], qp, s[1]); cmacr(o[2], qm, s[2]);
  o[3] = cscale(qa, s[1]); cmsub(o[3], qn, s[0]); cmacr(o[3], qm, s[3]);
}

template <class T> __device__ __forceinline__ void sdot_acc(cx<T>& c, const cx<T>* a, const cx<T>* b, bool neg) {
  if (neg) { cmsub(c, a[0], b[0]); cmsub(c, a[1], b[1]); cmsub(c, a[2], b[2]); cmsub(c, a[3], b[3]); }
  else { cmac(c, a[0], b[0]); cmac(c, a[1], b[1]); cmac(c, a[2], b[2]); cmac(c, a[3], b[3]); }
}

// quark current Jq^mu = ubar gamma^mu v
template <class T> __device__ __forceinline__ void quark_current(const cx<T>* u, const cx<T>* v, cx<T>* Jq) {
  // a = u[0..1], b = u[2..3], vL = v[0..1], vR = v[2..3]
  const cx<T> a0r0 = cmul(u[0], v[2]), a0r1 = cmul(u[0], v[3]), a1r0 = cmul(u[1], v[2]), a1r1 = cmul(u[1], v[3]);
  const cx<T> b0l0 = cmul(u[2], v[0]), b0l1 = cmul(u[2], v[1]), b1l0 = cmul(u[3], v[0]), b1l1 = cmul(u[3], v[1]);
  Jq[0] = {a0r0.r + a1r1.r + b0l0.r + b1l1.r, a0r0.i + a1r1.i + b0l0.i + b1l1.i};
  Jq[1] = {(a0r1.r + a1r0.r) - (b0l1.r + b1l0.r), (a0r1.i + a1r0.i) - (b0l1.i + b1l0.i)};
  const cx<T> t = {(a1r0.r - a0r1.r) - (b1l0.r - b0l1.r), (a1r0.i - a0r1.i) - (b1l0.i - b0l1.i)};
  Jq[2] = {-t.i, t.r};
  Jq[3] = {(a0r0.r - a1r1.r) - (b0l0.r - b1l1.r), (a0r0.i - a1r1.i) - (b0l0.i - b1l1.i)};
}

// colour sum of one helicity: sum_a A_a^* (sum_b Ctri_ab A_b), packed upper triangle
template <int NCOL, class T>
__device__ __forceinline__ T colour_sum(const cx<T>* A, const T* __restrict__ ctri) {
  T sum = 0;
  int idx = 0;
  for (int a = 0; a < NCOL; ++a) {
    T wr = 0, wi = 0;
    for (int b = a; b < NCOL; ++b, ++idx) {
      const T c = __ldg(ctri + idx);
      wr = fma(c, A[b].r, wr);
      wi = fma(c, A[b].i, wi);
    }
    sum = fma(A[a].r, wr, sum);
    sum = fma(A[a].i, wi, sum);
  }
  return sum;
}

// colour sum of one helicity from double-float jamps, evaluated in FP32 on their high parts (the
// quadratic form is well conditioned; the precision is needed in the jamps, not here)
template <int NCOL>
__device__ __forceinline__ float colour_sum_hi(const cx<dd::df>* A, const float* __restrict__ ctri) {
  float sum = 0.f;
  int idx = 0;
  for (int a = 0; a < NCOL; ++a) {
    float wr = 0.f, wi = 0.f;
    for (int b = a; b < NCOL; ++b, ++idx) {
      const float c = __ldg(ctri + idx);
      wr = fmaf(c, A[b].r.hi, wr);
      wi = fmaf(c, A[b].i.hi, wi);
    }
    sum = fmaf(A[a].r.hi, wr, sum);
    sum = fmaf(A[a].i.hi, wi, sum);
  }
  return sum;
}

// the colour table type of an amplitude type (FP32 integers for the double-float kernel)
template <class T> struct ColourT { using type = T; };
template <> struct ColourT<dd::df> { using type = float; };

// ---- per-event data shared by every helicity of an event (FP64 arithmetic, stored as T) ----
// Layout of one event's record (NITEM values of T): PT[S][4] (incoming gluon momentum of subset S),
// gprop[S] (-g/P_S^2), qc[S][5] (quark propagator coefficients), pol[g][5] (gluon polarisation basis,
// see gluon_pol), ubar[hel][4] complex, v[hel][4] complex (the NBASE items every record holds); then, in
// the FP32 record of 5 gluons, the currents of the gluon pairs (record_j2).  NITEM, the page stride.
template <int K> struct EvLayout {
  static constexpr int NSUB = 1 << K;
  static constexpr int PT = 0, GP = 4 * NSUB, QC = 5 * NSUB, EPS = 10 * NSUB, UB = EPS + 5 * K, VV = UB + 16;
  static constexpr int NBASE = VV + 16;
  static constexpr int NPAIR = K == 5 ? K * (K - 1) / 2 : 0;
  static constexpr int J2 = NBASE;
  static constexpr int NITEM = J2 + 32 * NPAIR;
};

// index of the gluon pair a < b among the K (K - 1) / 2 pairs in lexicographic order
__host__ __device__ constexpr int pair_index(int K, int a, int b) { return a * (2 * K - a - 1) / 2 + (b - a - 1); }

// The record in parts, each written through put(item, value): subsets S in [S0, S1) (S0 = 0 or 2^(K-1),
// so that every subset's momentum sum builds on one of the same range), the gluon polarisation bases,
// the top spinors.  A per-event kernel computes all parts; the fused FP32 kernel spreads them over warps.
template <int K, class T, int S0, int S1, class Put>
__device__ __forceinline__ void record_subsets(const double (*p)[4], const MeConst& cst, Put&& put) {
  using L = EvLayout<K>;
  static_assert(S0 == 0 || S0 == (1 << (K - 1)), "subset range");
  double Pst[S1 - S0][4];
#pragma unroll
  for (int S = S0; S < S1; ++S) {
    const int g = __ffs(S) - 1;
    const int part = g < 2 ? g : g + 2;
    const double sg = g < 2 ? 1.0 : -1.0;   // incoming gluons enter with +p, outgoing with -p
    if (S == 0) {
#pragma unroll
      for (int m = 0; m < 4; ++m) Pst[0][m] = 0.0;
    } else if ((S & (S - 1)) == 0 && S0 != 0) {
#pragma unroll
      for (int m = 0; m < 4; ++m) Pst[S - S0][m] = sg * p[part][m];
    } else {
#pragma unroll
      for (int m = 0; m < 4; ++m) Pst[S - S0][m] = Pst[(S & (S - 1)) - S0][m] + sg * p[part][m];
    }
  }
#pragma unroll
  for (int S = S0; S < S1; ++S) {
    const double* P = Pst[S - S0];
    if (S == 0 || S == (1 << K) - 1) {
      // the empty set and the set of all gluons: no current or quark-line prefix reads their momentum
      // sum or quark propagator; of the two, only the all-gluon propagator factor is read
      if (S != 0) {
        const double p2 = P[0] * P[0] - P[1] * P[1] - P[2] * P[2] - P[3] * P[3];
        put(L::GP + S, static_cast<T>(sizeof(T) == 8 ? -cst.gs / p2 : -cst.gs * rcp_nr(p2)));
      }
      continue;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) put(L::PT + 4 * S + m, static_cast<T>(P[m]));
    const double p2 = P[0] * P[0] - P[1] * P[1] - P[2] * P[2] - P[3] * P[3];
    const double Q0 = p[2][0] - P[0], Q1 = p[2][1] - P[1], Q2 = p[2][2] - P[2], Q3 = p[2][3] - P[3];
    const double dq = Q0 * Q0 - Q1 * Q1 - Q2 * Q2 - Q3 * Q3 - cst.mt * cst.mt;
    double gp, f;
    if constexpr (sizeof(T) == 8) {
      gp = (S & (S - 1)) ? -cst.gs / p2 : 0.0;   // includes one power of g
      f = -cst.gs / dq;
    } else {
      // FP32 amplitudes: the denominators P^2 and Q^2 - m^2 (where the cancellations are) and the
      // products in FP64, the reciprocals Newton-refined from FP32 seeds; one rounding to FP32 at the end
      gp = (S & (S - 1)) ? -cst.gs * rcp_nr(p2) : 0.0;
      f = -cst.gs * rcp_nr(dq);
    }
    put(L::GP + S, static_cast<T>(gp));
    put(L::QC + 5 * S + 0, static_cast<T>((Q0 + Q3) * f));
    put(L::QC + 5 * S + 1, static_cast<T>((Q0 - Q3) * f));
    put(L::QC + 5 * S + 2, static_cast<T>(Q1 * f));
    put(L::QC + 5 * S + 3, static_cast<T>(Q2 * f));
    put(L::QC + 5 * S + 4, static_cast<T>(cst.mt * f));
  }
}

template <int K, class T, class Put>
__device__ __forceinline__ void record_pols(const double (*p)[4], Put&& put) {
  using L = EvLayout<K>;
#pragma unroll
  for (int g = 0; g < K; ++g) {
    T pol[5];
    gluon_pol<T>(p[g < 2 ? g : g + 2], pol);
#pragma unroll
    for (int i = 0; i < 5; ++i) put(L::EPS + 5 * g + i, pol[i]);
  }
}

template <int K, class T, class Put>
__device__ __forceinline__ void record_tops(const double (*p)[4], const MeConst& cst, Put&& put) {
  using L = EvLayout<K>;
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    cx<T> ub[4], vv[4];
    top_ubar<T>(p[2], cst.mt, l ? 1 : -1, ub);
    top_v<T>(p[3], cst.mt, l ? 1 : -1, vv);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      put(L::UB + (l * 4 + a) * 2, ub[a].r);
      put(L::UB + (l * 4 + a) * 2 + 1, ub[a].i);
      put(L::VV + (l * 4 + a) * 2, vv[a].r);
      put(L::VV + (l * 4 + a) * 2 + 1, vv[a].i);
    }
  }
}

// FP32 record, 5 gluons: the current of every gluon pair a < b for the four helicity assignments h
// = h_a + 2 h_b (h = 1: helicity +1) of the pair, computed in FP64 and rounded once:
// J_ab = (-g / P_ab^2) V3(J_a, J_b; P_a, P_b), the canonical split of the length-2 sequence (a, b), with
// the incoming momenta of the pair's gluons.  Near a collinear pair the vertex numerator vanishes like
// sqrt(P_ab^2) while its terms do not, so its FP32 rounding, amplified by 1/P_ab^2, is a large part of the
// error of FP32 amplitudes near collinear pairs (measured: the FP32-kept events' largest error halves);
// the lane-group FP32 kernel takes these currents from the record instead.  Only for 5 gluons: there the
// 40 FP64 currents cost 0.3 % of an FP32 call; with 4 gluons their 24 cost 10 % (FP64 runs at 1/64 of the
// FP32 rate), more than the recomputations they save.
// Item J2 + ((pair_index(K, a, b) * 4 + h) * 4 + m) * 2 + (0: real, 1: imaginary part).
template <int K, class T, class Put>
__device__ __forceinline__ void record_j2(const double (*p)[4], const MeConst& cst, Put&& put) {
  using L = EvLayout<K>;
  double pol[K][5], P[K][4];
#pragma unroll
  for (int g = 0; g < K; ++g) {
    const int part = g < 2 ? g : g + 2;
    gluon_pol<double>(p[part], pol[g]);
#pragma unroll
    for (int m = 0; m < 4; ++m) P[g][m] = g < 2 ? p[part][m] : -p[part][m];
  }
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int b = a + 1; b < K; ++b) {
      const double P0 = P[a][0] + P[b][0], P1 = P[a][1] + P[b][1], P2 = P[a][2] + P[b][2], P3 = P[a][3] + P[b][3];
      const double gp = -cst.gs / (P0 * P0 - P1 * P1 - P2 * P2 - P3 * P3);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        cx<double> Ja[4], Jb[4], acc[4];
        ext_gluon(pol[a], (h & 1) ? 1 : -1, a >= 2, Ja);
        ext_gluon(pol[b], (h >> 1) ? 1 : -1, b >= 2, Jb);
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[m] = {0.0, 0.0};
        v3_acc(acc, Ja, Jb, P[a], P[b], false);
        const int base = L::J2 + (pair_index(K, a, b) * 4 + h) * 8;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          put(base + 2 * m, static_cast<T>(gp * acc[m].r));
          put(base + 2 * m + 1, static_cast<T>(gp * acc[m].i));
        }
      }
    }
}

template <int K, class T, class Put>
__device__ __forceinline__ void record_all(const double (*p)[4], const MeConst& cst, Put&& put) {
  record_subsets<K, T, 0, (1 << K)>(p, cst, put);
  record_pols<K, T>(p, put);
  record_tops<K, T>(p, cst, put);
}

// The whole record of one event as arrays (the kernels that compute it per thread)
template <int K, class T>
__device__ __forceinline__ void event_data(const double (*p)[4], const MeConst& cst, T (*PT)[4], T* gprop, T (*qc)[5],
                                           T (*pol)[5], cx<T> (*ub)[4], cx<T> (*vv)[4]) {
  using L = EvLayout<K>;
  T r[L::NBASE] = {};   // (the items no kernel reads stay zero)
  record_all<K, T>(p, cst, [&](int i, T v) { r[i] = v; });
  constexpr int NSUB = 1 << K;
#pragma unroll
  for (int S = 0; S < NSUB; ++S) {
#pragma unroll
    for (int m = 0; m < 4; ++m) PT[S][m] = r[L::PT + 4 * S + m];
    gprop[S] = r[L::GP + S];
#pragma unroll
    for (int c = 0; c < 5; ++c) qc[S][c] = r[L::QC + 5 * S + c];
  }
#pragma unroll
  for (int g = 0; g < K; ++g)
#pragma unroll
    for (int i = 0; i < 5; ++i) pol[g][i] = r[L::EPS + 5 * g + i];
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      ub[l][a] = {r[L::UB + (l * 4 + a) * 2], r[L::UB + (l * 4 + a) * 2 + 1]};
      vv[l][a] = {r[L::VV + (l * 4 + a) * 2], r[L::VV + (l * 4 + a) * 2 + 1]};
    }
}

// Smallest internal invariant of an event relative to s = (p1 + p2)^2: over the gluon propagators |P_S^2|
// (|S| >= 2) and the quark propagators |(p_t - P_S)^2 - m^2| (S neither empty nor all gluons), in FP32
// (absolute error ~1e-7 s, far below the thresholds it is compared with).
template <int K>
__device__ __forceinline__ float min_invariant_ratio(const double (*p)[4], float mt) {
  constexpr int NSUB = 1 << K;
  float q[K + 2][4];
#pragma unroll
  for (int i = 0; i < K + 2; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) q[i][m] = static_cast<float>(p[i][m]);
  float Pst[NSUB][4];
  float xmin = 3.0e38f;
#pragma unroll
  for (int m = 0; m < 4; ++m) Pst[0][m] = 0.f;
#pragma unroll
  for (int S = 1; S < NSUB; ++S) {
    const int g = __ffs(S) - 1;
    const int part = g < 2 ? g : g + 2;
    const float sg = g < 2 ? 1.f : -1.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) Pst[S][m] = Pst[S & (S - 1)][m] + sg * q[part][m];
    if (S == NSUB - 1) continue;
    const float* P = Pst[S];
    const float Q0 = q[2][0] - P[0], Q1 = q[2][1] - P[1], Q2 = q[2][2] - P[2], Q3 = q[2][3] - P[3];
    xmin = fminf(xmin, fabsf(Q0 * Q0 - Q1 * Q1 - Q2 * Q2 - Q3 * Q3 - mt * mt));
    if (S & (S - 1)) xmin = fminf(xmin, fabsf(P[0] * P[0] - P[1] * P[1] - P[2] * P[2] - P[3] * P[3]));
  }
  const float s0 = q[0][0] + q[1][0], s1 = q[0][1] + q[1][1], s2 = q[0][2] + q[1][2], s3 = q[0][3] + q[1][3];
  return xmin / fabsf(s0 * s0 - s1 * s1 - s2 * s2 - s3 * s3);
}

}  // namespace v2
}  // namespace mg
