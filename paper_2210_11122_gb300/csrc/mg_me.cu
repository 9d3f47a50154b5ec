// mg_me.cu -- per-event, per-helicity matrix elements of g g -> t tbar + (K-2) g on the device.
//
// Hot path of the paper (Sec. 2): for every phase-space point and helicity the kernel builds
// the external wavefunctions (HELAS conventions: circular gluon polarisations, massive helicity
// spinors for t and tbar), sums every tree Feynman diagram into colour-ordered amplitudes
// ("jamps", one per colour flow), forms the colour quadratic form A^dagger C A and sums the
// helicities that survived the helicity filter.  Feynman-gauge QCD vertices (quark-gluon
// i g gamma^mu T^a; three- and four-gluon vertices) are organised as the colour-ordered
// Berends-Giele recursion of mg_tables.cpp; the colour matrix is exact (mg_colour.cpp).
//
// Thread mapping: one thread per (event, good helicity); a warp covers 32 consecutive events of
// one AoSoA page, so every momentum load of a warp is one 256-byte line.  The per-(event,
// helicity) colour sums go to out[slot][event] and a second kernel adds the helicities in a
// fixed order (bit-reproducible FP64 sums).
#include <cuda_runtime.h>

#include "mg_internal.h"
#include "mg_kernels.h"

namespace mg {

template <class T>
struct cx {
  T r, i;
};
template <class T> __device__ __forceinline__ cx<T> C(T r, T i) { return cx<T>{r, i}; }
template <class T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.r + b.r, a.i + b.i}; }
template <class T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.r - b.r, a.i - b.i}; }
template <class T> __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
template <class T> __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return {s * a.r, s * a.i}; }
template <class T> __device__ __forceinline__ cx<T> cneg(cx<T> a) { return {-a.r, -a.i}; }
template <class T> __device__ __forceinline__ cx<T> cconj(cx<T> a) { return {a.r, -a.i}; }
template <class T> __device__ __forceinline__ cx<T> mul_i(cx<T> a) { return {-a.i, a.r}; }

// Minkowski products (+,-,-,-), no conjugation
template <class T> __device__ __forceinline__ cx<T> mdot(const cx<T>* a, const cx<T>* b) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
template <class T> __device__ __forceinline__ cx<T> mdot(const cx<T>* a, const T* p) {
  return {a[0].r * p[0] - a[1].r * p[1] - a[2].r * p[2] - a[3].r * p[3],
          a[0].i * p[0] - a[1].i * p[1] - a[2].i * p[2] - a[3].i * p[3]};
}

template <int K> struct Sizes;
template <> struct Sizes<2> { static constexpr int ncol = 2, nseq = 2, nfull = 1; };
template <> struct Sizes<3> { static constexpr int ncol = 6, nseq = 6, nfull = 3; };
template <> struct Sizes<4> { static constexpr int ncol = 24, nseq = 22, nfull = 12; };
template <> struct Sizes<5> { static constexpr int ncol = 120, nseq = 105, nfull = 60; };

__device__ __forceinline__ int ref_slot(int16_t r) { return r >> 1; }
__device__ __forceinline__ bool ref_neg(int16_t r) { return r & 1; }

// ---------------------------------------------------------------------------------------
// External wavefunctions (double precision; chiral representation, spinors ordered
// (left pair; right pair)).
// ---------------------------------------------------------------------------------------
// Helicity eigenspinor chi_lam of the direction of p (sigma.p^ chi = lam chi); for p along -z
// the theta -> pi limit at phi = 0 is used.
__device__ __forceinline__ void chi2(const double* p, int lam, cx<double>* c) {
  const double px = p[1], py = p[2], pz = p[3];
  const double pt2 = px * px + py * py;
  const double pa = sqrt(pt2 + pz * pz);
  const double apz = pz >= 0.0 ? pa + pz : pt2 / (pa - pz);   // |p| + pz without cancellation
  if (apz > 0.0) {
    const double n = rsqrt(2.0 * pa * apz);
    if (lam > 0) { c[0] = C(apz * n, 0.0); c[1] = C(px * n, py * n); }
    else { c[0] = C(-px * n, py * n); c[1] = C(apz * n, 0.0); }
  } else {
    if (lam > 0) { c[0] = C(0.0, 0.0); c[1] = C(1.0, 0.0); }
    else { c[0] = C(-1.0, 0.0); c[1] = C(0.0, 0.0); }
  }
}

// outgoing quark: ubar = (u_R^*, u_L^*), u_L = sqrt(E - lam|p|) chi, u_R = sqrt(E + lam|p|) chi
__device__ __forceinline__ void ext_ubar(const double* p, double m, int lam, cx<double>* w) {
  const double pa = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  const double sp = sqrt(p[0] + pa);
  const double sm = m > 0.0 ? m / sp : 0.0;
  cx<double> c[2];
  chi2(p, lam, c);
  const double fl = lam > 0 ? sm : sp, fr = lam > 0 ? sp : sm;
  w[0] = cconj(fr * c[0]); w[1] = cconj(fr * c[1]);
  w[2] = cconj(fl * c[0]); w[3] = cconj(fl * c[1]);
}

// outgoing antiquark of helicity lam: v = (-lam sqrt(E + lam|p|) chi_{-lam}; lam sqrt(E - lam|p|) chi_{-lam})
__device__ __forceinline__ void ext_v(const double* p, double m, int lam, cx<double>* w) {
  const double pa = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  const double sp = sqrt(p[0] + pa);
  const double sm = m > 0.0 ? m / sp : 0.0;
  cx<double> c[2];
  chi2(p, -lam, c);
  const double fl = lam > 0 ? -sp : sm, fr = lam > 0 ? sm : -sp;
  w[0] = fl * c[0]; w[1] = fl * c[1];
  w[2] = fr * c[0]; w[3] = fr * c[1];
}

// gluon: eps(k, lam) = (0, (-lam e_theta - i e_phi)/sqrt 2), conjugated for an outgoing gluon
__device__ __forceinline__ void ext_eps(const double* k, int lam, bool outgoing, cx<double>* w) {
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
  w[0] = C(0.0, 0.0);
#pragma unroll
  for (int i = 0; i < 3; ++i) w[1 + i] = C(sl * et[i], si * ep[i]);
}

// ---------------------------------------------------------------------------------------
// Spinor algebra (T = double or float)
// ---------------------------------------------------------------------------------------
// row spinor s times gamma.J: (a, b) [[0, J.sigma], [J.sigmabar, 0]] = (b J.sigmabar, a J.sigma)
template <class T> __device__ __forceinline__ void row_gamma(const cx<T>* s, const cx<T>* J, cx<T>* o) {
  const cx<T> jm = {J[1].r + J[2].i, J[1].i - J[2].r};   // J1 - i J2
  const cx<T> jp = {J[1].r - J[2].i, J[1].i + J[2].r};   // J1 + i J2
  const cx<T> a = J[0] + J[3], b = J[0] - J[3];
  o[0] = s[2] * a + s[3] * jp;
  o[1] = s[2] * jm + s[3] * b;
  o[2] = s[0] * b - s[1] * jp;
  o[3] = s[1] * a - s[0] * jm;
}

// column: (gamma.J) v = (J.sigma v_R ; J.sigmabar v_L)
template <class T> __device__ __forceinline__ void gamma_col(const cx<T>* J, const cx<T>* v, cx<T>* o) {
  const cx<T> jm = {J[1].r + J[2].i, J[1].i - J[2].r};
  const cx<T> jp = {J[1].r - J[2].i, J[1].i + J[2].r};
  const cx<T> a = J[0] + J[3], b = J[0] - J[3];
  o[0] = b * v[2] - jm * v[3];
  o[1] = a * v[3] - jp * v[2];
  o[2] = a * v[0] + jm * v[1];
  o[3] = jp * v[0] + b * v[1];
}

// row spinor times (Qslash + m), Q real
template <class T> __device__ __forceinline__ void row_slash_m(const cx<T>* s, const T* Q, T m, cx<T>* o) {
  const cx<T> qm = {Q[1], -Q[2]}, qp = {Q[1], Q[2]};
  const T a = Q[0] + Q[3], b = Q[0] - Q[3];
  o[0] = a * s[2] + s[3] * qp + m * s[0];
  o[1] = s[2] * qm + b * s[3] + m * s[1];
  o[2] = b * s[0] - s[1] * qp + m * s[2];
  o[3] = a * s[1] - s[0] * qm + m * s[3];
}

template <class T> __device__ __forceinline__ cx<T> sdot(const cx<T>* a, const cx<T>* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
}

// ---------------------------------------------------------------------------------------
// The kernel: one thread = one (event, helicity).
// ---------------------------------------------------------------------------------------
template <int K, class T>
__global__ void __launch_bounds__(kMeThreads)
k_me_helicity(const double* __restrict__ mom, int64_t nevt, const Tables* __restrict__ tab,
              const int* __restrict__ hels, const int* __restrict__ nslot_dev, const double* __restrict__ ctri,
              MeConst cst, double* __restrict__ out, int64_t out_stride) {
  constexpr int npar = K + 2;
  constexpr int NSEQ = Sizes<K>::nseq;
  constexpr int NCOL = Sizes<K>::ncol;
  constexpr int NFULL = Sizes<K>::nfull;
  constexpr int NSUB = 1 << K;
  const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int slot = blockIdx.y;
  if (e >= nevt || slot >= *nslot_dev) return;
  const int h = hels[slot];

  // ---- momenta (AoSoA) ----
  double p[npar][4];
  {
    const double* base = mom + (e / kPage) * npar * 4 * kPage + (e % kPage);
#pragma unroll
    for (int i = 0; i < npar; ++i)
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) p[i][mu] = __ldg(base + (i * 4 + mu) * kPage);
  }
  auto lam = [&](int i) { return ((h >> (npar - 1 - i)) & 1) ? 1 : -1; };

  // ---- incoming gluon momenta and subset sums (double), propagator factors ----
  double P[NSUB][4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) P[0][mu] = 0.0;
#pragma unroll
  for (int S = 1; S < NSUB; ++S) {
    const int g = __ffs(S) - 1;
    const int part = g < 2 ? g : g + 2;
    const double sg = g < 2 ? 1.0 : -1.0;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) P[S][mu] = P[S & (S - 1)][mu] + sg * p[part][mu];
  }
  T PT[NSUB][4];
  T gprop[NSUB];       // -1/P^2 of a gluon current over subset S (|S| >= 2)
  cx<T> qfac[NSUB];    // -g / (Q^2 - m^2 + i m w), Q = p_t - P(S), for quark lines
#pragma unroll
  for (int S = 0; S < NSUB; ++S) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) PT[S][mu] = static_cast<T>(P[S][mu]);
    const double p2 = P[S][0] * P[S][0] - P[S][1] * P[S][1] - P[S][2] * P[S][2] - P[S][3] * P[S][3];
    gprop[S] = static_cast<T>(S && (S & (S - 1)) ? -1.0 / p2 : 0.0);
    double Q[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) Q[mu] = p[2][mu] - P[S][mu];
    const double dre = Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3] - cst.mt * cst.mt;
    const double dim = cst.mt * cst.wt;
    const double nrm = -cst.gs / (dre * dre + dim * dim);
    qfac[S] = C(static_cast<T>(dre * nrm), static_cast<T>(-dim * nrm));
  }

  // ---- external wavefunctions ----
  cx<T> J[NSEQ][4];
  cx<T> ub[4], vv[4];
  {
    cx<double> w[4];
#pragma unroll
    for (int g = 0; g < K; ++g) {
      const int part = g < 2 ? g : g + 2;
      ext_eps(p[part], lam(part), g >= 2, w);
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) J[g][mu] = C(static_cast<T>(w[mu].r), static_cast<T>(w[mu].i));
    }
    ext_ubar(p[2], cst.mt, lam(2), w);
#pragma unroll
    for (int a = 0; a < 4; ++a) ub[a] = C(static_cast<T>(w[a].r), static_cast<T>(w[a].i));
    ext_v(p[3], cst.mt, lam(3), w);
#pragma unroll
    for (int a = 0; a < 4; ++a) vv[a] = C(static_cast<T>(w[a].r), static_cast<T>(w[a].i));
  }
  const T gs = static_cast<T>(cst.gs);

  // ---- gluon currents of canonical sequences, by increasing length ----
  for (int s = K; s < NSEQ; ++s) {
    const int S = tab->seq_mask[s];
    cx<T> a3[4] = {}, a4[4] = {};
    const int n3 = tab->seq_nv3[s];
    for (int k = 0; k < n3; ++k) {
      const int16_t rl = tab->seq_v3[s][k][0], rr = tab->seq_v3[s][k][1];
      const cx<T>* JL = J[ref_slot(rl)];
      const cx<T>* JR = J[ref_slot(rr)];
      const T* PL = PT[tab->seq_mask[ref_slot(rl)]];
      const T* PR = PT[tab->seq_mask[ref_slot(rr)]];
      T d[4], u1[4], u2[4];
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) { d[mu] = PL[mu] - PR[mu]; u1[mu] = PL[mu] + 2 * PR[mu]; u2[mu] = 2 * PL[mu] + PR[mu]; }
      const cx<T> jj = mdot(JL, JR), cl = mdot(JL, u1), cr = mdot(JR, u2);
      const T sg = (ref_neg(rl) != ref_neg(rr)) ? T(-1) : T(1);
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) a3[mu] = a3[mu] + sg * (d[mu] * jj + cl * JR[mu] - cr * JL[mu]);
    }
    const int n4 = tab->seq_nv4[s];
    for (int k = 0; k < n4; ++k) {
      const int16_t ra = tab->seq_v4[s][k][0], rb = tab->seq_v4[s][k][1], rc = tab->seq_v4[s][k][2];
      const cx<T>* JA = J[ref_slot(ra)];
      const cx<T>* JB = J[ref_slot(rb)];
      const cx<T>* JC = J[ref_slot(rc)];
      const cx<T> ab = mdot(JA, JB), bc = mdot(JB, JC), ac = mdot(JA, JC);
      const T sg = (ref_neg(ra) ^ ref_neg(rb) ^ ref_neg(rc)) ? T(-1) : T(1);
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) a4[mu] = a4[mu] + sg * (ab * JC[mu] + bc * JA[mu] - T(2) * (ac * JB[mu]));
    }
    const T f3 = gprop[S] * gs, f4 = gprop[S] * gs * gs;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) J[s][mu] = f3 * a3[mu] + f4 * a4[mu];
  }

  // ---- quark-antiquark current Jq^mu = ubar gamma^mu v; X = (gamma.J) v; D = J.Jq ----
  cx<T> Jq[4];
  {
    // a = ubar[0..1], b = ubar[2..3], vL = v[0..1], vR = v[2..3]
    const cx<T> avr0 = ub[0] * vv[2], avr1 = ub[0] * vv[3], a1vr0 = ub[1] * vv[2], a1vr1 = ub[1] * vv[3];
    const cx<T> bvl0 = ub[2] * vv[0], bvl1 = ub[2] * vv[1], b1vl0 = ub[3] * vv[0], b1vl1 = ub[3] * vv[1];
    Jq[0] = avr0 + a1vr1 + bvl0 + b1vl1;
    Jq[1] = (avr1 + a1vr0) - (bvl1 + b1vl0);
    Jq[2] = mul_i((a1vr0 - avr1) - (b1vl0 - bvl1));
    Jq[3] = (avr0 - a1vr1) - (bvl0 - b1vl1);
  }
  cx<T> X[NSEQ][4];
  cx<T> D[NSEQ];
  for (int s = 0; s < NSEQ; ++s) {
    gamma_col(J[s], vv, X[s]);
    D[s] = sdot(ub, X[s]);
  }

  // ---- all gluons on one current attached to the quark line (canonical orderings) ----
  cx<T> F[NFULL];
  {
    const double* Pa = P[NSUB - 1];
    const T gfull = static_cast<T>(-1.0 / (Pa[0] * Pa[0] - Pa[1] * Pa[1] - Pa[2] * Pa[2] - Pa[3] * Pa[3]));
    for (int f = 0; f < NFULL; ++f) {
      cx<T> s3 = {}, s4 = {};
      const int n3 = tab->full_nv3[f];
      for (int k = 0; k < n3; ++k) {
        const int16_t rl = tab->full_v3[f][k][0], rr = tab->full_v3[f][k][1];
        const int il = ref_slot(rl), ir = ref_slot(rr);
        const T* PL = PT[tab->seq_mask[il]];
        const T* PR = PT[tab->seq_mask[ir]];
        T d[4], u1[4], u2[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) { d[mu] = PL[mu] - PR[mu]; u1[mu] = PL[mu] + 2 * PR[mu]; u2[mu] = 2 * PL[mu] + PR[mu]; }
        const cx<T> t = mdot(J[il], J[ir]) * mdot(Jq, d) + mdot(J[il], u1) * D[ir] - mdot(J[ir], u2) * D[il];
        s3 = s3 + ((ref_neg(rl) != ref_neg(rr)) ? cneg(t) : t);
      }
      const int n4 = tab->full_nv4[f];
      for (int k = 0; k < n4; ++k) {
        const int16_t ra = tab->full_v4[f][k][0], rb = tab->full_v4[f][k][1], rc = tab->full_v4[f][k][2];
        const int ia = ref_slot(ra), ib = ref_slot(rb), ic = ref_slot(rc);
        const cx<T> t = mdot(J[ia], J[ib]) * D[ic] + mdot(J[ib], J[ic]) * D[ia] - T(2) * (mdot(J[ia], J[ic]) * D[ib]);
        s4 = s4 + ((ref_neg(ra) ^ ref_neg(rb) ^ ref_neg(rc)) ? cneg(t) : t);
      }
      F[f] = gfull * (gs * s3 + (gs * gs) * s4);
    }
  }

  // ---- depth-first walk over the colour orderings: quark-line prefixes and jamps ----
  cx<T> A[NCOL];
  cx<T> stk[K][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) stk[0][a] = ub[a];
  const T mt = static_cast<T>(cst.mt);
  for (int c = 0; c < NCOL; ++c) {
    const int l = tab->lcp[c];
    for (int m = (l > 0 ? l : 0) + 1; m < K; ++m) {
      cx<T> acc[4] = {};
      for (int j = 0; j < m; ++j) {
        const int16_t r = tab->sub[c][j][m];
        cx<T> t[4];
        row_gamma(stk[j], J[ref_slot(r)], t);
        if (ref_neg(r)) {
#pragma unroll
          for (int a = 0; a < 4; ++a) acc[a] = acc[a] - t[a];
        } else {
#pragma unroll
          for (int a = 0; a < 4; ++a) acc[a] = acc[a] + t[a];
        }
      }
      const int S = tab->prefix_mask[c][m];
      T Q[4];
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) Q[mu] = static_cast<T>(p[2][mu] - P[S][mu]);
      cx<T> t[4];
      row_slash_m(acc, Q, mt, t);
#pragma unroll
      for (int a = 0; a < 4; ++a) stk[m][a] = t[a] * qfac[S];
    }
    const int fi = tab->full_idx[c];
    cx<T> amp = fi >= 0 ? F[fi] : ((K & 1) ? F[-fi - 1] : cneg(F[-fi - 1]));   // (-1)^(K+1) under reflection
    for (int j = 1; j < K; ++j) {
      const int16_t r = tab->sub[c][j][K];
      const cx<T> t = sdot(stk[j], X[ref_slot(r)]);
      amp = ref_neg(r) ? amp - t : amp + t;
    }
    A[c] = amp;
  }

  // ---- colour sum A^dagger C A (packed upper triangle, off-diagonal entries doubled) ----
  T sum = 0;
  int idx = 0;
  for (int a = 0; a < NCOL; ++a) {
    T row = 0;
    for (int b = a; b < NCOL; ++b, ++idx) {
      const T cab = static_cast<T>(__ldg(ctri + idx));
      row += cab * (A[a].r * A[b].r + A[a].i * A[b].i);
    }
    sum += row;
  }
  out[slot * out_stride + e] = static_cast<double>(sum) * cst.colour_scale;
}

// me[e] = norm * sum_slot out[slot][e], fixed order
__global__ void k_hel_sum(const double* __restrict__ part, const int* __restrict__ nslot_dev, int64_t nevt,
                          int64_t stride, double norm, double* __restrict__ me) {
  const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (e >= nevt) return;
  const int nslot = *nslot_dev;
  double s = 0.0;
  for (int k = 0; k < nslot; ++k) s += part[k * stride + e];
  me[e] = s * norm;
}

// helicity filter, step 1: maxr[h] = max over the warm-up events of part[h][e] / tot[e]
// (one block per helicity, fixed-shape tree reduction: order-independent maximum).
__global__ void k_hel_ratio_max(const double* __restrict__ part, const double* __restrict__ tot, int64_t nevt,
                                int64_t stride, double* __restrict__ maxr) {
  __shared__ double red[256];
  const int h = blockIdx.x;
  double mx = 0.0;
  for (int64_t e = threadIdx.x; e < nevt; e += blockDim.x) {
    const double r = part[h * stride + e] / tot[e];
    mx = r > mx ? r : mx;
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = red[threadIdx.x + w] > red[threadIdx.x] ? red[threadIdx.x + w] : red[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) maxr[h] = red[0];
}

// step 2: good(h) <=> maxr[h] > tau; mask words, ascending good list and its length.
__global__ void k_hel_mask(const double* __restrict__ maxr, int nhel, double tau, uint32_t* __restrict__ mask,
                           int* __restrict__ good, int* __restrict__ ngood) {
  const int h = threadIdx.x;
  const bool g = h < nhel && maxr[h] > tau;
  const unsigned bits = __ballot_sync(0xffffffffu, g);
  if ((h & 31) == 0 && h < ((nhel + 31) & ~31)) mask[h >> 5] = bits;
  __syncthreads();
  if (h == 0) {
    int n = 0;
    for (int k = 0; k < nhel; ++k)
      if ((mask[k >> 5] >> (k & 31)) & 1u) good[n++] = k;
    *ngood = n;
  }
}

template <int K, class T>
static cudaError_t launch_me_t(const double* mom, int64_t nevt, const Tables* tab, const int* hels, int maxslot,
                               const int* nslot, const double* ctri, const MeConst& cst, double* out, int64_t stride,
                               cudaStream_t st) {
  dim3 grid(static_cast<unsigned>((nevt + kMeThreads - 1) / kMeThreads), static_cast<unsigned>(maxslot));
  if (grid.x == 0 || grid.y == 0) return cudaSuccess;
  { k_me_helicity<K, T><<<grid, kMeThreads, 0, st>>>(mom, nevt, tab, hels, nslot, ctri, cst, out, stride); mg::note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_me_helicity(int K, bool fp32, const double* mom, int64_t nevt, const Tables* tab, const int* hels,
                               int maxslot, const int* nslot, const double* ctri, const MeConst& cst, double* out,
                               int64_t stride, cudaStream_t st) {
  switch (K * 2 + (fp32 ? 1 : 0)) {
    case 4: return launch_me_t<2, double>(mom, nevt, tab, hels, maxslot, nslot, ctri, cst, out, stride, st);
    case 5: return launch_me_t<2, float>(mom, nevt, tab, hels, maxslot, nslot, ctri, cst, out, stride, st);
    case 6: return launch_me_t<3, double>(mom, nevt, tab, hels, maxslot, nslot, ctri, cst, out, stride, st);
    case 7: return launch_me_t<3, float>(mom, nevt, tab, hels, maxslot, nslot, ctri, cst, out, stride, st);
    case 8: return launch_me_t<4, double>(mom, nevt, tab, hels, maxslot, nslot, ctri, cst, out, stride, st);
    case 9: return launch_me_t<4, float>(mom, nevt, tab, hels, maxslot, nslot, ctri, cst, out, stride, st);
    case 10: return launch_me_t<5, double>(mom, nevt, tab, hels, maxslot, nslot, ctri, cst, out, stride, st);
    case 11: return launch_me_t<5, float>(mom, nevt, tab, hels, maxslot, nslot, ctri, cst, out, stride, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_hel_sum(const double* part, const int* nslot, int64_t nevt, int64_t stride, double norm,
                           double* me, cudaStream_t st) {
  const int threads = 256;
  const unsigned blocks = static_cast<unsigned>((nevt + threads - 1) / threads);
  if (blocks == 0) return cudaSuccess;
  { k_hel_sum<<<blocks, threads, 0, st>>>(part, nslot, nevt, stride, norm, me); mg::note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_hel_mask(const double* part, const double* tot, int nhel, int64_t nevt, int64_t stride, double tau,
                            double* maxr, uint32_t* mask, int* good, int* ngood, cudaStream_t st) {
  { k_hel_ratio_max<<<nhel, 256, 0, st>>>(part, tot, nevt, stride, maxr); mg::note_launch(); }
  { k_hel_mask<<<1, 128, 0, st>>>(maxr, nhel, tau, mask, good, ngood); mg::note_launch(); }
  return cudaGetLastError();
}

}  // namespace mg
