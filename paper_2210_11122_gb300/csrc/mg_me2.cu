// mg_me2.cu -- matrix-element kernel, one thread per (event, gluon-helicity combination).
//
// Same physics as the per-helicity kernel of mg_me.cu (HELAS wavefunctions, every tree diagram of
// g g -> t tbar + (K-2) g summed into colour-ordered amplitudes by the Berends-Giele recursion of
// mg_tables.cpp, exact colour matrix, helicity sum; the hot path of the paper's Sec. 2), organised
// for GB300's FP64 pipe (2 DFMA/clk/SM, 1/64 of FP32), where the instruction count is the cost:
//   * the gluon currents J(seq) and the all-gluon currents J(sigma) depend only on the gluon
//     helicities: one thread computes them once and reuses them for the 4 top-helicity pairs;
//   * quark-line prefixes depend on the top helicity only: one depth-first walk per top helicity,
//     each leaf forming the amplitudes of both antitop helicities;
//   * (gamma.J) v is precomputed per antitop helicity for every gluon current;
//   * every complex product-accumulate is an FMA chain; the quark propagator factor
//     -g/(Q^2 - m^2) is folded into the coefficients of (Qslash + m) once per event subset.
// Output: per slot (gluon combination) the colour-summed |M_h|^2 summed over its good top
// helicities, or (filter mode) |M_h|^2 of every helicity h separately.
#include <cuda_runtime.h>

#include "mg_internal.h"
#include "mg_kernels.h"

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

// ---- external wavefunctions (FP64) ----
__device__ __forceinline__ void chi2(const double* p, int lam, cx<double>* c) {
  const double px = p[1], py = p[2], pz = p[3];
  const double pt2 = px * px + py * py;
  const double pa = sqrt(pt2 + pz * pz);
  const double apz = pz >= 0.0 ? pa + pz : pt2 / (pa - pz);
  if (apz > 0.0) {
    const double n = rsqrt(2.0 * pa * apz);
    if (lam > 0) { c[0] = {apz * n, 0.0}; c[1] = {px * n, py * n}; }
    else { c[0] = {-px * n, py * n}; c[1] = {apz * n, 0.0}; }
  } else {
    if (lam > 0) { c[0] = {0.0, 0.0}; c[1] = {1.0, 0.0}; }
    else { c[0] = {-1.0, 0.0}; c[1] = {0.0, 0.0}; }
  }
}

template <class T>
__device__ __forceinline__ void top_ubar(const double* p, double m, int lam, cx<T>* w) {
  const double pa = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  const double sp = sqrt(p[0] + pa);
  const double sm = m > 0.0 ? m / sp : 0.0;
  cx<double> c[2];
  chi2(p, lam, c);
  const double fl = lam > 0 ? sm : sp, fr = lam > 0 ? sp : sm;
  w[0] = {T(fr * c[0].r), T(-fr * c[0].i)}; w[1] = {T(fr * c[1].r), T(-fr * c[1].i)};
  w[2] = {T(fl * c[0].r), T(-fl * c[0].i)}; w[3] = {T(fl * c[1].r), T(-fl * c[1].i)};
}

template <class T>
__device__ __forceinline__ void top_v(const double* p, double m, int lam, cx<T>* w) {
  const double pa = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  const double sp = sqrt(p[0] + pa);
  const double sm = m > 0.0 ? m / sp : 0.0;
  cx<double> c[2];
  chi2(p, -lam, c);
  const double fl = lam > 0 ? -sp : sm, fr = lam > 0 ? sm : -sp;
  w[0] = {T(fl * c[0].r), T(fl * c[0].i)}; w[1] = {T(fl * c[1].r), T(fl * c[1].i)};
  w[2] = {T(fr * c[0].r), T(fr * c[0].i)}; w[3] = {T(fr * c[1].r), T(fr * c[1].i)};
}

template <class T>
__device__ __forceinline__ void gluon_eps(const double* k, int lam, bool outgoing, cx<T>* w) {
  const double kx = k[1], ky = k[2], kz = k[3];
  const double kt = sqrt(kx * kx + ky * ky);
  const double ka = sqrt(kx * kx + ky * ky + kz * kz);
  double et[3], ep[3];
  if (kt > 0.0) {
    const double inv = 1.0 / (ka * kt);
    et[0] = kx * kz * inv; et[1] = ky * kz * inv; et[2] = -kt / ka;
    ep[0] = -ky / kt; ep[1] = kx / kt; ep[2] = 0.0;
  } else {
    et[0] = kz < 0.0 ? -1.0 : 1.0; et[1] = 0.0; et[2] = 0.0;
    ep[0] = 0.0; ep[1] = 1.0; ep[2] = 0.0;
  }
  const double r = 0.70710678118654752440;
  const double sl = lam > 0 ? -r : r;
  const double si = outgoing ? r : -r;
  w[0] = {T(0), T(0)};
#pragma unroll
  for (int i = 0; i < 3; ++i) w[1 + i] = {T(sl * et[i]), T(si * ep[i])};
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

// acc (+/-)= s gamma.J  (row spinor s, gluon current J)
template <class T>
__device__ __forceinline__ void row_gamma_acc(cx<T>* acc, const cx<T>* s, const cx<T>* J, bool neg) {
  cx<T> jm = {J[1].r + J[2].i, J[1].i - J[2].r};   // J1 - i J2
  cx<T> jp = {J[1].r - J[2].i, J[1].i + J[2].r};   // J1 + i J2
  cx<T> a = {J[0].r + J[3].r, J[0].i + J[3].i}, b = {J[0].r - J[3].r, J[0].i - J[3].i};
  if (neg) { jm = cneg(jm); jp = cneg(jp); a = cneg(a); b = cneg(b); }
  cmac(acc[0], s[2], a); cmac(acc[0], s[3], jp);
  cmac(acc[1], s[2], jm); cmac(acc[1], s[3], b);
  cmac(acc[2], s[0], b); cmsub(acc[2], s[1], jp);
  cmac(acc[3], s[1], a); cmsub(acc[3], s[0], jm);
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

// ---- per-event data shared by every helicity of an event (FP64 arithmetic, stored as T) ----
// Layout of one event's record (NITEM values of T): PT[S][4] (incoming gluon momentum of subset S),
// gprop[S] (-g/P_S^2), qc[S][5] (quark propagator coefficients), eps[g][hel][4] complex,
// ubar[hel][4] complex, v[hel][4] complex.
template <int K> struct EvLayout {
  static constexpr int NSUB = 1 << K;
  static constexpr int PT = 0, GP = 4 * NSUB, QC = 5 * NSUB, EPS = 10 * NSUB, UB = EPS + 16 * K, VV = UB + 16;
  static constexpr int NITEM = VV + 16;
};

template <int K, class T>
__device__ __forceinline__ void event_data(const double (*p)[4], const MeConst& cst, T (*PT)[4], T* gprop, T (*qc)[5],
                                           cx<T> (*eps)[2][4], cx<T> (*ub)[4], cx<T> (*vv)[4],
                                           double* min_invariant = nullptr) {
  constexpr int NSUB = 1 << K;
  double xmin = 1e300;
  double Pst[NSUB][4];
#pragma unroll
  for (int m = 0; m < 4; ++m) Pst[0][m] = 0.0;
#pragma unroll
  for (int S = 1; S < NSUB; ++S) {
    const int g = __ffs(S) - 1;
    const int part = g < 2 ? g : g + 2;
    const double sg = g < 2 ? 1.0 : -1.0;
#pragma unroll
    for (int m = 0; m < 4; ++m) Pst[S][m] = Pst[S & (S - 1)][m] + sg * p[part][m];
  }
#pragma unroll
  for (int S = 0; S < NSUB; ++S) {
    const double* P = Pst[S];
#pragma unroll
    for (int m = 0; m < 4; ++m) PT[S][m] = static_cast<T>(P[m]);
    const double p2 = P[0] * P[0] - P[1] * P[1] - P[2] * P[2] - P[3] * P[3];
    gprop[S] = static_cast<T>((S & (S - 1)) ? -cst.gs / p2 : 0.0);   // includes one power of g
    const double Q0 = p[2][0] - P[0], Q1 = p[2][1] - P[1], Q2 = p[2][2] - P[2], Q3 = p[2][3] - P[3];
    const double dq = Q0 * Q0 - Q1 * Q1 - Q2 * Q2 - Q3 * Q3 - cst.mt * cst.mt;
    const double f = -cst.gs / dq;
    if (S != 0 && S != NSUB - 1) {   // internal lines only (S = 0 and S = all are the external tops)
      xmin = fmin(xmin, fabs(dq));
      if (S & (S - 1)) xmin = fmin(xmin, fabs(p2));
    }
    qc[S][0] = static_cast<T>((Q0 + Q3) * f);
    qc[S][1] = static_cast<T>((Q0 - Q3) * f);
    qc[S][2] = static_cast<T>(Q1 * f);
    qc[S][3] = static_cast<T>(Q2 * f);
    qc[S][4] = static_cast<T>(cst.mt * f);
  }
#pragma unroll
  for (int g = 0; g < K; ++g) {
    const int part = g < 2 ? g : g + 2;
    gluon_eps<T>(p[part], -1, g >= 2, eps[g][0]);
    gluon_eps<T>(p[part], 1, g >= 2, eps[g][1]);
  }
  top_ubar<T>(p[2], cst.mt, -1, ub[0]);
  top_ubar<T>(p[2], cst.mt, 1, ub[1]);
  top_v<T>(p[3], cst.mt, -1, vv[0]);
  top_v<T>(p[3], cst.mt, 1, vv[1]);
  if (min_invariant) {
    const double s0 = p[0][0] + p[1][0], s1 = p[0][1] + p[1][1], s2 = p[0][2] + p[1][2], s3 = p[0][3] + p[1][3];
    const double shat = s0 * s0 - s1 * s1 - s2 * s2 - s3 * s3;   // (p1 + p2)^2
    *min_invariant = xmin / fabs(shat);
  }
}

// One thread per event: the event's record, AoSoA (page of 32 events, value-major within a page).
// repair != NULL: events whose smallest internal invariant |P^2| or |Q^2 - m^2| (over the gluon and
// quark propagators of the recursion) is below cst.fp32_tau * s are appended to repair[] (count in
// *nrepair): FP32 rounding is amplified ~ 1/sqrt(invariant/s) there (collinear and soft gluons).
template <int K, class T>
__global__ void __launch_bounds__(128) k_event_prep(const double* __restrict__ mom, int64_t nevt, MeConst cst,
                                                    T* __restrict__ rec, int* __restrict__ repair,
                                                    int* __restrict__ nrepair) {
  constexpr int npar = K + 2, NSUB = 1 << K;
  using L = EvLayout<K>;
  const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (e >= nevt) return;
  double p[npar][4];
  const double* base = mom + (e / kPage) * npar * 4 * kPage + (e % kPage);
#pragma unroll
  for (int i = 0; i < npar; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) p[i][m] = __ldg(base + (i * 4 + m) * kPage);
  T PT[NSUB][4], gprop[NSUB], qc[NSUB][5];
  cx<T> eps[K][2][4], ub[2][4], vv[2][4];
  double xmin = 1.0;
  event_data<K, T>(p, cst, PT, gprop, qc, eps, ub, vv, &xmin);
  if (repair && xmin < cst.fp32_tau) repair[atomicAdd(nrepair, 1)] = static_cast<int>(e);
  T* out = rec + (e / kPage) * L::NITEM * kPage + (e % kPage);
#pragma unroll
  for (int S = 0; S < NSUB; ++S) {
#pragma unroll
    for (int m = 0; m < 4; ++m) out[(L::PT + 4 * S + m) * kPage] = PT[S][m];
    out[(L::GP + S) * kPage] = gprop[S];
#pragma unroll
    for (int c = 0; c < 5; ++c) out[(L::QC + 5 * S + c) * kPage] = qc[S][c];
  }
#pragma unroll
  for (int g = 0; g < K; ++g)
#pragma unroll
    for (int l = 0; l < 2; ++l)
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        out[(L::EPS + ((g * 2 + l) * 4 + m) * 2) * kPage] = eps[g][l][m].r;
        out[(L::EPS + ((g * 2 + l) * 4 + m) * 2 + 1) * kPage] = eps[g][l][m].i;
      }
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      out[(L::UB + (l * 4 + a) * 2) * kPage] = ub[l][a].r;
      out[(L::UB + (l * 4 + a) * 2 + 1) * kPage] = ub[l][a].i;
      out[(L::VV + (l * 4 + a) * 2) * kPage] = vv[l][a].r;
      out[(L::VV + (l * 4 + a) * 2 + 1) * kPage] = vv[l][a].i;
    }
}

// JOUT: instead of colour sums, write the jamps of every helicity of the slot as FP32 complex
// numbers to jout[((e * 4 * 2^K) + slot * 4 + 2 * top + antitop) * ncol + sigma] (zeros for helicities
// outside the mask), for the tensor-core colour sum.
template <int K, class T, bool PER_HEL, bool PREP, bool JOUT>
__global__ void __launch_bounds__(kMeThreads)
k_me_gluonhel(const double* __restrict__ mom, const T* __restrict__ rec, int64_t nevt, const Tables* __restrict__ tab,
              const int* __restrict__ gslots, const int* __restrict__ nslot_dev, const uint32_t* __restrict__ mask,
              const T* __restrict__ ctri, MeConst cst, double* __restrict__ out, int64_t stride,
              float2* __restrict__ jout, int tile_ev, int slot_major, const int* __restrict__ evlist,
              const int* __restrict__ nlist, int rows_out) {
  constexpr int npar = K + 2;
  constexpr int NSEQ = Sizes<K>::nseq;
  constexpr int NCOL = Sizes<K>::ncol;
  constexpr int NFULL = Sizes<K>::nfull;
  constexpr int NSUB = 1 << K;
  const int tile_sl = kMeThreads / tile_ev;
  const unsigned bev = slot_major ? blockIdx.y : blockIdx.x, bsl = slot_major ? blockIdx.x : blockIdx.y;
  const int64_t et = static_cast<int64_t>(bev) * tile_ev + threadIdx.x % tile_ev;
  const int slot = static_cast<int>(bsl) * tile_sl + static_cast<int>(threadIdx.x) / tile_ev;
  if (et >= nevt || slot >= *nslot_dev) return;
  // evlist: the thread works on event evlist[et] of the batch (et < *nlist), else on event et
  if (evlist && et >= *nlist) return;
  const int64_t e = evlist ? static_cast<int64_t>(evlist[et]) : et;
  const int gc = gslots[slot];   // bit g = helicity (+1) of gluon g

  const T gs = static_cast<T>(cst.gs);
  T PT[NSUB][4];
  T gprop[NSUB];
  T qc[NSUB][5];
  cx<T> J[NSEQ][4];
  cx<T> ub[2][4], vv[2][4];
  if (PREP) {
    using L = EvLayout<K>;
    const T* in = rec + (e / kPage) * L::NITEM * kPage + (e % kPage);
#pragma unroll
    for (int S = 0; S < NSUB; ++S) {
#pragma unroll
      for (int m = 0; m < 4; ++m) PT[S][m] = __ldg(in + (L::PT + 4 * S + m) * kPage);
      gprop[S] = __ldg(in + (L::GP + S) * kPage);
#pragma unroll
      for (int c = 0; c < 5; ++c) qc[S][c] = __ldg(in + (L::QC + 5 * S + c) * kPage);
    }
#pragma unroll
    for (int g = 0; g < K; ++g) {
      const int l = (gc >> g) & 1;
#pragma unroll
      for (int m = 0; m < 4; ++m)
        J[g][m] = {__ldg(in + (L::EPS + ((g * 2 + l) * 4 + m) * 2) * kPage),
                   __ldg(in + (L::EPS + ((g * 2 + l) * 4 + m) * 2 + 1) * kPage)};
    }
#pragma unroll
    for (int l = 0; l < 2; ++l)
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        ub[l][a] = {__ldg(in + (L::UB + (l * 4 + a) * 2) * kPage), __ldg(in + (L::UB + (l * 4 + a) * 2 + 1) * kPage)};
        vv[l][a] = {__ldg(in + (L::VV + (l * 4 + a) * 2) * kPage), __ldg(in + (L::VV + (l * 4 + a) * 2 + 1) * kPage)};
      }
  } else {
    double p[npar][4];
    const double* base = mom + (e / kPage) * npar * 4 * kPage + (e % kPage);
#pragma unroll
    for (int i = 0; i < npar; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) p[i][m] = __ldg(base + (i * 4 + m) * kPage);
    cx<T> eps[K][2][4];
    event_data<K, T>(p, cst, PT, gprop, qc, eps, ub, vv);
#pragma unroll
    for (int g = 0; g < K; ++g)
#pragma unroll
      for (int m = 0; m < 4; ++m) J[g][m] = eps[g][(gc >> g) & 1][m];
  }

  // ---- gluon currents (helicities of gc) ----
  for (int s = K; s < NSEQ; ++s) {
    cx<T> acc[4] = {};
    const int n3 = tab->seq_nv3[s];
    for (int k = 0; k < n3; ++k) {
      const int16_t rl = tab->seq_v3[s][k][0], rr = tab->seq_v3[s][k][1];
      const int il = rslot(rl), ir = rslot(rr);
      v3_acc(acc, J[il], J[ir], PT[tab->seq_mask[il]], PT[tab->seq_mask[ir]], rneg(rl) != rneg(rr));
    }
    const int n4 = tab->seq_nv4[s];
    for (int k = 0; k < n4; ++k) {
      const int16_t ra = tab->seq_v4[s][k][0], rb = tab->seq_v4[s][k][1], rc = tab->seq_v4[s][k][2];
      v4_acc(acc, J[rslot(ra)], J[rslot(rb)], J[rslot(rc)], gs, rneg(ra) ^ rneg(rb) ^ rneg(rc));
    }
    const T f = gprop[tab->seq_mask[s]];
#pragma unroll
    for (int m = 0; m < 4; ++m) J[s][m] = cscale(f, acc[m]);
  }
  // all gluons on one current (canonical orderings)
  cx<T> JF[NFULL][4];
  for (int f = 0; f < NFULL; ++f) {
    cx<T> acc[4] = {};
    const int n3 = tab->full_nv3[f];
    for (int k = 0; k < n3; ++k) {
      const int16_t rl = tab->full_v3[f][k][0], rr = tab->full_v3[f][k][1];
      const int il = rslot(rl), ir = rslot(rr);
      v3_acc(acc, J[il], J[ir], PT[tab->seq_mask[il]], PT[tab->seq_mask[ir]], rneg(rl) != rneg(rr));
    }
    const int n4 = tab->full_nv4[f];
    for (int k = 0; k < n4; ++k) {
      const int16_t ra = tab->full_v4[f][k][0], rb = tab->full_v4[f][k][1], rc = tab->full_v4[f][k][2];
      v4_acc(acc, J[rslot(ra)], J[rslot(rb)], J[rslot(rc)], gs, rneg(ra) ^ rneg(rb) ^ rneg(rc));
    }
    const T fz = gprop[NSUB - 1];
#pragma unroll
    for (int m = 0; m < 4; ++m) JF[f][m] = cscale(fz, acc[m]);
  }

  // ---- antitop spinors and (gamma.J) v for both antitop helicities ----
  // (gamma.J) v for every current and both antitop helicities: precomputed in FP64 (saves FP64
  // instructions); in FP32 each jamp term forms ubar-side (row spinor x gamma.J) on the fly instead,
  // keeping 2 NSEQ spinors out of the thread's local memory (FP32 arithmetic is cheap, memory is not).
  constexpr bool kTableX = sizeof(T) == 8;
  cx<T> X[kTableX ? 2 : 1][kTableX ? NSEQ : 1][4];
  if (kTableX) {
#pragma unroll
    for (int b = 0; b < 2; ++b)
      for (int s = 0; s < NSEQ; ++s) gamma_col(J[s], vv[b], X[b][s]);
  }

  // helicity index of (gc, top helicity a, antitop helicity b)
  int hbase = 0;
#pragma unroll
  for (int g = 0; g < K; ++g)
    if ((gc >> g) & 1) hbase |= 1 << (npar - 1 - (g < 2 ? g : g + 2));
  const int bit_t = 1 << (npar - 3), bit_tb = 1 << (npar - 4);

  double total = 0.0;
  for (int a = 0; a < 2; ++a) {
    const int h0 = hbase | (a ? bit_t : 0), h1 = h0 | bit_tb;
    const bool good0 = PER_HEL || ((mask[h0 >> 5] >> (h0 & 31)) & 1u);
    const bool good1 = PER_HEL || ((mask[h1 >> 5] >> (h1 & 31)) & 1u);
    if (!good0 && !good1) {
      if (JOUT) {
        float2* row = jout + (e * (4 << K) + slot * 4 + 2 * a) * NCOL;
        for (int c = 0; c < 2 * NCOL; ++c) row[c] = make_float2(0.f, 0.f);
      }
      continue;
    }
    cx<T> stk[K][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) stk[0][q] = ub[a][q];
    cx<T> Jq[2][4];
    quark_current(stk[0], vv[0], Jq[0]);
    quark_current(stk[0], vv[1], Jq[1]);
    cx<T> A[2][NCOL];
    for (int c = 0; c < NCOL; ++c) {
      const int l = tab->lcp[c];
      for (int m = l + 1; m < K; ++m) {
        cx<T> acc[4] = {};
        for (int j = 0; j < m; ++j) {
          const int16_t r = tab->sub[c][j][m];
          row_gamma_acc(acc, stk[j], J[rslot(r)], rneg(r));
        }
        row_prop(acc, qc[tab->prefix_mask[c][m]], stk[m]);
      }
      const int fi = tab->full_idx[c];
      const int fidx = fi >= 0 ? fi : -fi - 1;
      const bool fneg = fi < 0 && !(K & 1);   // reflection sign (-1)^(K+1)
      if (kTableX) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          cx<T> amp = mdot(Jq[b], JF[fidx]);   // all gluons on one current: ubar gamma.J v = Jq.J
          if (fneg) amp = cneg(amp);
          for (int j = 1; j < K; ++j) {
            const int16_t r = tab->sub[c][j][K];
            sdot_acc(amp, stk[j], X[b][rslot(r)], rneg(r));
          }
          A[b][c] = amp;
        }
      } else {
        cx<T> amp0 = mdot(Jq[0], JF[fidx]), amp1 = mdot(Jq[1], JF[fidx]);
        if (fneg) { amp0 = cneg(amp0); amp1 = cneg(amp1); }
        for (int j = 1; j < K; ++j) {
          const int16_t r = tab->sub[c][j][K];
          cx<T> t[4] = {};
          row_gamma_acc(t, stk[j], J[rslot(r)], rneg(r));
          sdot_acc(amp0, t, vv[0], false);
          sdot_acc(amp1, t, vv[1], false);
        }
        A[0][c] = amp0;
        A[1][c] = amp1;
      }
    }
    if (JOUT) {
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const bool good = b ? good1 : good0;
        float2* row = jout + (e * (4 << K) + slot * 4 + 2 * a + b) * NCOL;
        for (int c = 0; c < NCOL; ++c)
          row[c] = good ? make_float2(static_cast<float>(A[b][c].r), static_cast<float>(A[b][c].i)) : make_float2(0.f, 0.f);
      }
      continue;
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int h = b ? h1 : h0;
      const bool good = b ? good1 : good0;
      if (!good) continue;
      const double v = static_cast<double>(colour_sum<NCOL, T>(A[b], ctri)) * cst.colour_scale;
      if (PER_HEL) out[h * stride + e] = v;
      else total += v;
    }
  }
  if (!PER_HEL && !JOUT) {
    if (rows_out) {   // tensor-core row layout: slot*4 + (2 top + antitop); the slot total in the first row
      out[(slot * 4) * stride + e] = total;
      out[(slot * 4 + 1) * stride + e] = 0.0;
      out[(slot * 4 + 2) * stride + e] = 0.0;
      out[(slot * 4 + 3) * stride + e] = 0.0;
    } else {
      out[slot * stride + e] = total;
    }
  }
}

// Gluon-helicity combinations with at least one good helicity (fixed ascending order).
__global__ void k_gluon_slots(const uint32_t* __restrict__ mask, int K, int* __restrict__ gslots, int* __restrict__ n,
                              int* __restrict__ nrows) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int npar = K + 2;
  int cnt = 0;
  for (int gc = 0; gc < (1 << K); ++gc) {
    int hb = 0;
    for (int g = 0; g < K; ++g)
      if ((gc >> g) & 1) hb |= 1 << (npar - 1 - (g < 2 ? g : g + 2));
    bool any = false;
    for (int t = 0; t < 4; ++t) {
      const int h = hb | ((t & 1) << (npar - 3)) | ((t >> 1) << (npar - 4));
      any = any || ((mask[h >> 5] >> (h & 31)) & 1u);
    }
    if (any) gslots[cnt++] = gc;
  }
  *n = cnt;
  *nrows = 4 * cnt;
}

}  // namespace v2

cudaError_t launch_gluon_slots(const uint32_t* mask, int K, int* gslots, int* n, int* nrows, cudaStream_t st) {
  v2::k_gluon_slots<<<1, 32, 0, st>>>(mask, K, gslots, n, nrows);
  return cudaGetLastError();
}

template <int K, class T, bool PER_HEL>
static cudaError_t launch_v2(const double* mom, void* prep, int64_t nevt, const Tables* tab, const int* gslots,
                             int maxslot, const int* nslot, const uint32_t* mask, const void* ctri_any,
                             const MeConst& cst, double* out, int64_t stride, float2* jout, MeShape shape,
                             int* repair, int* nrepair, const int* evlist, const int* nlist, int rows_out,
                             cudaStream_t st) {
  const T* ctri = static_cast<const T*>(ctri_any);
  int tev = shape.tile_ev;
  if (tev != 32 && tev != 64 && tev != 128) tev = 128;
  const int tsl = kMeThreads / tev;
  const unsigned nev_t = static_cast<unsigned>((nevt + tev - 1) / tev), nsl_t = static_cast<unsigned>((maxslot + tsl - 1) / tsl);
  const int sm = shape.slot_major ? 1 : 0;
  dim3 grid = sm ? dim3(nsl_t, nev_t) : dim3(nev_t, nsl_t);
  if (nev_t == 0 || nsl_t == 0) return cudaSuccess;
  if (prep && !PER_HEL) {
    T* rec = static_cast<T*>(prep);
    v2::k_event_prep<K, T><<<static_cast<unsigned>((nevt + 127) / 128), 128, 0, st>>>(mom, nevt, cst, rec, repair,
                                                                                     nrepair);
    if (jout)
      v2::k_me_gluonhel<K, T, false, true, true><<<grid, kMeThreads, 0, st>>>(mom, rec, nevt, tab, gslots, nslot, mask,
                                                                             ctri, cst, out, stride, jout, tev, sm, nullptr, nullptr, 0);
    else
      v2::k_me_gluonhel<K, T, false, true, false><<<grid, kMeThreads, 0, st>>>(mom, rec, nevt, tab, gslots, nslot,
                                                                              mask, ctri, cst, out, stride, nullptr, tev,
                                                                              sm, nullptr, nullptr, 0);
  } else {
    v2::k_me_gluonhel<K, T, PER_HEL, false, false><<<grid, kMeThreads, 0, st>>>(mom, nullptr, nevt, tab, gslots, nslot,
                                                                                 mask, ctri, cst, out, stride, nullptr,
                                                                                 tev, sm, evlist, nlist, rows_out);
  }
  return cudaGetLastError();
}

int64_t event_record_bytes(int K, bool fp32) {
  int nitem = 0;
  switch (K) {
    case 2: nitem = v2::EvLayout<2>::NITEM; break;
    case 3: nitem = v2::EvLayout<3>::NITEM; break;
    case 4: nitem = v2::EvLayout<4>::NITEM; break;
    case 5: nitem = v2::EvLayout<5>::NITEM; break;
    default: return 0;
  }
  return static_cast<int64_t>(nitem) * (fp32 ? 4 : 8);
}

cudaError_t launch_me_gluonhel(int K, bool fp32, bool per_hel, const double* mom, void* prep, int64_t nevt,
                               const Tables* tab, const int* gslots, int maxslot, const int* nslot,
                               const uint32_t* mask, const double* ctri64, const float* ctri32, const MeConst& cst,
                               double* out, int64_t stride, cudaStream_t st, float2* jout, MeShape shape,
                               int* repair, int* nrepair, const int* evlist, const int* nlist, int rows_out) {
#define MG_V2_CASE(KK)                                                                                              \
  case KK:                                                                                                          \
    if (per_hel) return fp32 ? launch_v2<KK, float, true>(mom, prep, nevt, tab, gslots, maxslot, nslot, mask, ctri32, cst,  \
                                                          out, stride, jout, shape, repair, nrepair, evlist, nlist, rows_out, st)                                          \
                             : launch_v2<KK, double, true>(mom, prep, nevt, tab, gslots, maxslot, nslot, mask, ctri64, cst, \
                                                           out, stride, jout, shape, repair, nrepair, evlist, nlist, rows_out, st);                                        \
    return fp32 ? launch_v2<KK, float, false>(mom, prep, nevt, tab, gslots, maxslot, nslot, mask, ctri32, cst, out, stride, \
                                              jout, shape, repair, nrepair, evlist, nlist, rows_out, st)                                                                   \
                : launch_v2<KK, double, false>(mom, prep, nevt, tab, gslots, maxslot, nslot, mask, ctri64, cst, out, stride,\
                                               jout, shape, repair, nrepair, evlist, nlist, rows_out, st);
  switch (K) {
    MG_V2_CASE(2)
    MG_V2_CASE(3)
    MG_V2_CASE(4)
    MG_V2_CASE(5)
    default: return cudaErrorInvalidValue;
  }
#undef MG_V2_CASE
}

}  // namespace mg
