// me_oracle.cpp -- TEST INFRASTRUCTURE ONLY.
//
// Plain, slow, FP64 CPU oracle for the per-event tree-level QCD matrix element of
// g g -> t tbar + n_g gluons (n_g = 0..3), following the workflow of arXiv 2210.11122
// (Sec. 1 and Fig. 1: random numbers -> phase-space momenta -> matrix element per event;
// Sec. 2: the matrix element is the hot path).  The paper prints no formulas; every step
// below is written from the textbook definition it names:
//
//   * Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
//     1, 2, 3", SC'11 (round function, multipliers and Weyl key schedule).
//   * RAMBO: Kleiss, Stirling, Ellis, Comput. Phys. Commun. 40 (1986) 359 (massless
//     momenta, then the massive rescaling with its weight).
//   * Wavefunctions: helicity spinors and circular polarisation vectors in the chiral
//     representation (HELAS conventions, Murayama-Watanabe-Hagiwara KEK-91-11).
//   * Amplitudes: Feynman-gauge QCD Feynman rules (Peskin-Schroeder Sec. 16.1 conventions:
//     quark vertex i g gamma^mu T^a, three-gluon vertex g f^abc V^{mu nu rho}, four-gluon
//     vertex -i g^2 [f f ...], gluon propagator -i g_{mu nu}/k^2, quark propagator
//     i(pslash+m)/(p^2-m^2)), organised as a Berends-Giele recursion (Nucl. Phys. B306
//     (1988) 759) over colour-ordered currents (Mangano-Parke, Phys. Rep. 200 (1991) 301).
//     With one quark line, M = sum_sigma (T^{a_sigma1}...T^{a_sigmak})_{i_t j_tbar} A(sigma)
//     holds exactly (each f^{abc} = -i Tr-commutator, no 1/N terms).
//   * Colour sum: sum_colours |M|^2 = sum_{sigma,tau} A(sigma) C(sigma,tau) A(tau)^*, with
//     the exact colour matrix C passed in by the caller (oracle/colour.py).
//
// Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may load
// this library.  It shares no code with the CUDA path.
//
// Conventions (stated once, used throughout):
//   metric (+,-,-,-); momenta (E,px,py,pz); particle order g1, g2, t, tbar, g3, g4, g5;
//   incoming p1 = (sqrt(s)/2)(1,0,0,1), p2 = (sqrt(s)/2)(1,0,0,-1);
//   helicity index h = sum_i bit_i 2^(npar-1-i), bit_i = 1 for lambda_i = +1, particle 0 is
//   the most significant bit; helicity labels are physical helicities;
//   gluon labels 0..k-1 are the gluons in particle order (g1, g2, g3, ...), k = n_g + 2;
//   jamp index = rank of sigma among the permutations of (0..k-1) in lexicographic order.

#include <cstdint>
#include <cmath>
#include <cstring>
#include <vector>
#include <thread>
#include <algorithm>

namespace {

// ------------------------------------------------------------------------------------
// Flop-counting scalar.  Every +,-,* counts one flop; / and sqrt are counted separately.
// A complex multiply therefore counts 6 (4 mul + 2 add) and a complex add 2.
// ------------------------------------------------------------------------------------
struct Counter { unsigned long long add, mul, div, sqrt; };
thread_local Counter tl_count = {0, 0, 0, 0};

struct Cd {
  double v;
  Cd() : v(0) {}
  Cd(double x) : v(x) {}
};
inline Cd operator+(Cd a, Cd b) { tl_count.add++; return Cd(a.v + b.v); }
inline Cd operator-(Cd a, Cd b) { tl_count.add++; return Cd(a.v - b.v); }
inline Cd operator*(Cd a, Cd b) { tl_count.mul++; return Cd(a.v * b.v); }
inline Cd operator/(Cd a, Cd b) { tl_count.div++; return Cd(a.v / b.v); }
inline Cd operator-(Cd a) { return Cd(-a.v); }
inline bool operator>(Cd a, Cd b) { return a.v > b.v; }
inline bool operator<(Cd a, Cd b) { return a.v < b.v; }
inline bool operator>=(Cd a, Cd b) { return a.v >= b.v; }
inline Cd sqrt(Cd a) { tl_count.sqrt++; return Cd(std::sqrt(a.v)); }
inline double val(Cd a) { return a.v; }
inline double val(double a) { return a; }

using std::sqrt;

template <class R> struct Cx {
  R re, im;
  Cx() : re(0.0), im(0.0) {}
  Cx(R r, R i) : re(r), im(i) {}
};
template <class R> inline Cx<R> operator+(const Cx<R>& a, const Cx<R>& b) { return Cx<R>(a.re + b.re, a.im + b.im); }
template <class R> inline Cx<R> operator-(const Cx<R>& a, const Cx<R>& b) { return Cx<R>(a.re - b.re, a.im - b.im); }
template <class R> inline Cx<R> operator*(const Cx<R>& a, const Cx<R>& b) {
  return Cx<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R> inline Cx<R> scale(R s, const Cx<R>& a) { return Cx<R>(s * a.re, s * a.im); }
template <class R> inline Cx<R> conj(const Cx<R>& a) { return Cx<R>(a.re, -a.im); }
template <class R> inline Cx<R> times_i(const Cx<R>& a) { return Cx<R>(-a.im, a.re); }   // i*a

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al. SC'11): 10 rounds of the 4x32 S-box with multipliers
// 0xD2511F53, 0xCD9E8D57; the key is bumped by the Weyl constants 0x9E3779B9,
// 0xBB67AE85 between rounds.
// ------------------------------------------------------------------------------------
void philox4x32_10(const uint32_t in[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = in[0], x1 = in[1], x2 = in[2], x3 = in[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// Uniforms for (event e, final-state particle j): counter {e_lo, e_hi, j, 0},
// key {seed_lo, seed_hi}; u = (x + 0.5) * 2^-32, exact in FP64 and strictly inside (0,1).
void event_uniforms(uint64_t seed, uint64_t e, uint32_t j, double u[4]) {
  uint32_t ctr[4] = {(uint32_t)e, (uint32_t)(e >> 32), j, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  philox4x32_10(ctr, key, x);
  for (int i = 0; i < 4; ++i) u[i] = ((double)x[i] + 0.5) * 0x1p-32;
}

double factorial(int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

// ------------------------------------------------------------------------------------
// RAMBO (Kleiss-Stirling-Ellis).  n final-state particles, uniforms u[n][4].
// Returns 0 on success, 1 if the massive Newton solve did not converge, 2 if
// sqrt(s) <= sum of masses.
// ------------------------------------------------------------------------------------
int rambo(int n, const double* masses, const double* u, double sqrts, double* p, double* wgt) {
  const double pi = 3.14159265358979323846;
  double msum = 0;
  for (int i = 0; i < n; ++i) msum += masses[i];
  if (!(sqrts > msum)) return 2;
  // massless stage: isotropic q_i with energy density q0 exp(-q0)
  std::vector<double> q(4 * n);
  double Q[4] = {0, 0, 0, 0};
  for (int i = 0; i < n; ++i) {
    const double* r = u + 4 * i;
    double c = 2.0 * r[0] - 1.0;
    double s = std::sqrt(1.0 - c * c);
    double f = 2.0 * pi * r[1];
    double q0 = -std::log(r[2] * r[3]);
    q[4 * i + 0] = q0;
    q[4 * i + 1] = q0 * s * std::cos(f);
    q[4 * i + 2] = q0 * s * std::sin(f);
    q[4 * i + 3] = q0 * c;
    for (int m = 0; m < 4; ++m) Q[m] += q[4 * i + m];
  }
  // conformal transformation onto total momentum (sqrt(s), 0, 0, 0)
  double M = std::sqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
  double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
  double gam = Q[0] / M;
  double a = 1.0 / (1.0 + gam);
  double x = sqrts / M;
  for (int i = 0; i < n; ++i) {
    const double* qi = &q[4 * i];
    double bq = b[0] * qi[1] + b[1] * qi[2] + b[2] * qi[3];
    p[4 * i + 0] = x * (gam * qi[0] + bq);
    for (int m = 0; m < 3; ++m) p[4 * i + 1 + m] = x * (qi[1 + m] + b[m] * qi[0] + a * bq * b[m]);
  }
  // massless flat weight
  double w = std::pow(2.0 * pi, 4 - 3 * n) * std::pow(pi / 2.0, n - 1) * std::pow(sqrts * sqrts, n - 2) /
             (factorial(n - 1) * factorial(n - 2));
  if (msum == 0.0) { *wgt = w; return 0; }
  // massive stage: solve sum_i sqrt(m_i^2 + xi^2 E_i^2) = sqrt(s) by Newton's method
  double xi = std::sqrt(1.0 - (msum / sqrts) * (msum / sqrts));
  int converged = 0;
  for (int it = 0; it < 50; ++it) {
    double f = -sqrts, fp = 0;
    for (int i = 0; i < n; ++i) {
      double e = std::sqrt(masses[i] * masses[i] + xi * xi * p[4 * i] * p[4 * i]);
      f += e;
      fp += xi * p[4 * i] * p[4 * i] / e;
    }
    if (std::fabs(f) <= 1e-14 * sqrts) { converged = 1; break; }
    xi -= f / fp;
  }
  double prodv = 1.0, sumv = 0.0;
  for (int i = 0; i < n; ++i) {
    double e = std::sqrt(masses[i] * masses[i] + xi * xi * p[4 * i] * p[4 * i]);
    double v = xi * p[4 * i];  // |k_i| = xi |p_i| = xi E_i for the massless p_i
    for (int m = 1; m < 4; ++m) p[4 * i + m] *= xi;
    p[4 * i] = e;
    prodv *= v / e;
    sumv += v * v / e;
  }
  w *= std::pow(xi, 2 * n - 3) * prodv * sqrts / sumv;
  *wgt = w;
  return converged ? 0 : 1;
}

// ------------------------------------------------------------------------------------
// External wavefunctions (chiral representation, gamma^mu = [[0, sigma^mu],[sigmabar^mu, 0]],
// spinor = (left-handed pair; right-handed pair)).
// ------------------------------------------------------------------------------------
// Two-component helicity eigenspinor chi_lam(p^): (sigma.p^) chi = lam chi.
template <class R> void helicity_chi(const R* p3, int lam, Cx<R> chi[2]) {
  R px = p3[0], py = p3[1], pz = p3[2];
  R pt2 = px * px + py * py;
  R pp = sqrt(pt2 + pz * pz);
  // pp + pz, written without cancellation for pz < 0
  R ppz = (pz >= R(0.0)) ? pp + pz : pt2 / (pp - pz);
  if (ppz > R(0.0)) {
    R nrm = R(1.0) / sqrt(R(2.0) * pp * ppz);
    if (lam > 0) {
      chi[0] = Cx<R>(ppz * nrm, R(0.0));
      chi[1] = Cx<R>(px * nrm, py * nrm);
    } else {
      chi[0] = Cx<R>(-px * nrm, py * nrm);
      chi[1] = Cx<R>(ppz * nrm, R(0.0));
    }
  } else {  // p along -z: theta = pi, phi = 0
    if (lam > 0) { chi[0] = Cx<R>(); chi[1] = Cx<R>(R(1.0), R(0.0)); }
    else { chi[0] = Cx<R>(R(-1.0), R(0.0)); chi[1] = Cx<R>(); }
  }
}

// Outgoing fermion: ubar(p, lam) = u^dagger gamma^0, u = (sqrt(E - lam|p|) chi_lam ; sqrt(E + lam|p|) chi_lam).
template <class R> void wf_ubar(const R* p, R m, int lam, Cx<R> out[4]) {
  R pp = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  R wp = sqrt(p[0] + pp);                      // sqrt(E + |p|)
  R wm = (m * m > R(0.0)) ? m / wp : R(0.0);   // sqrt(E - |p|) = m / sqrt(E + |p|)
  Cx<R> chi[2];
  helicity_chi(p + 1, lam, chi);
  R wL = (lam > 0) ? wm : wp;   // u_L = sqrt(E - lam|p|) chi
  R wR = (lam > 0) ? wp : wm;   // u_R = sqrt(E + lam|p|) chi
  // ubar = (u_R^*, u_L^*)
  out[0] = conj(scale(wR, chi[0]));
  out[1] = conj(scale(wR, chi[1]));
  out[2] = conj(scale(wL, chi[0]));
  out[3] = conj(scale(wL, chi[1]));
}

// Outgoing antifermion of physical helicity lam:
// v(p, lam) = (-lam sqrt(E + lam|p|) chi_{-lam} ; lam sqrt(E - lam|p|) chi_{-lam}).
template <class R> void wf_v(const R* p, R m, int lam, Cx<R> out[4]) {
  R pp = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  R wp = sqrt(p[0] + pp);
  R wm = (m * m > R(0.0)) ? m / wp : R(0.0);
  Cx<R> chi[2];
  helicity_chi(p + 1, -lam, chi);
  R wL = (lam > 0) ? -wp : wm;   // -lam sqrt(E + lam|p|)
  R wR = (lam > 0) ? wm : -wp;   //  lam sqrt(E - lam|p|)
  out[0] = scale(wL, chi[0]);
  out[1] = scale(wL, chi[1]);
  out[2] = scale(wR, chi[0]);
  out[3] = scale(wR, chi[1]);
}

// Circular polarisation epsilon^mu(k, lam) = (0, (-lam e_theta - i e_phi)/sqrt(2)).
template <class R> void wf_eps(const R* k, int lam, Cx<R> e[4]) {
  R kx = k[1], ky = k[2], kz = k[3];
  R kt = sqrt(kx * kx + ky * ky);
  R kk = sqrt(kx * kx + ky * ky + kz * kz);
  R eth[3], eph[3];
  if (kt > R(0.0)) {
    eth[0] = kx * kz / (kk * kt); eth[1] = ky * kz / (kk * kt); eth[2] = -kt / kk;
    eph[0] = -ky / kt; eph[1] = kx / kt; eph[2] = R(0.0);
  } else {  // along +z or -z, phi = 0
    eth[0] = (kz < R(0.0)) ? R(-1.0) : R(1.0); eth[1] = R(0.0); eth[2] = R(0.0);
    eph[0] = R(0.0); eph[1] = R(1.0); eph[2] = R(0.0);
  }
  R r2 = R(1.0) / sqrt(R(2.0));
  R sl = (lam > 0) ? -r2 : r2;
  e[0] = Cx<R>();
  for (int i = 0; i < 3; ++i) e[1 + i] = Cx<R>(sl * eth[i], -r2 * eph[i]);
}

// ------------------------------------------------------------------------------------
// Lorentz algebra on complex vectors (contravariant components).
// ------------------------------------------------------------------------------------
template <class R> Cx<R> dot_cc(const Cx<R>* a, const Cx<R>* b) {   // a.b, no conjugation
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
template <class R> Cx<R> dot_cr(const Cx<R>* a, const R* p) {
  return Cx<R>(a[0].re * p[0] - a[1].re * p[1] - a[2].re * p[2] - a[3].re * p[3],
               a[0].im * p[0] - a[1].im * p[1] - a[2].im * p[2] - a[3].im * p[3]);
}
template <class R> R dot_rr(const R* a, const R* b) { return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]; }

// Row spinor times gamma.J (J complex, contravariant):
// gamma.J = [[0, J.sigma],[J.sigmabar, 0]], J.sigma = J0 - sigma.J, J.sigmabar = J0 + sigma.J.
// (a, b) gamma.J = (b (J.sigmabar), a (J.sigma)).
template <class R> void row_gamma(const Cx<R>* s, const Cx<R>* J, Cx<R>* out) {
  Cx<R> i1(R(0.0), R(1.0));
  Cx<R> Jm = J[1] - i1 * J[2];   // J1 - i J2
  Cx<R> Jp = J[1] + i1 * J[2];   // J1 + i J2
  // J.sigmabar = [[J0+J3, Jm],[Jp, J0-J3]]
  Cx<R> sb00 = J[0] + J[3], sb01 = Jm, sb10 = Jp, sb11 = J[0] - J[3];
  // J.sigma = [[J0-J3, -Jm],[-Jp, J0+J3]]
  Cx<R> s00 = J[0] - J[3], s01 = Cx<R>() - Jm, s10 = Cx<R>() - Jp, s11 = J[0] + J[3];
  out[0] = s[2] * sb00 + s[3] * sb10;
  out[1] = s[2] * sb01 + s[3] * sb11;
  out[2] = s[0] * s00 + s[1] * s10;
  out[3] = s[0] * s01 + s[1] * s11;
}
// Row spinor times (Qslash + m), Q real.
template <class R> void row_qslash_plus_m(const Cx<R>* s, const R* Q, R m, Cx<R>* out) {
  Cx<R> J[4];
  for (int i = 0; i < 4; ++i) J[i] = Cx<R>(Q[i], R(0.0));
  row_gamma(s, J, out);
  for (int i = 0; i < 4; ++i) out[i] = out[i] + scale(m, s[i]);
}

// ------------------------------------------------------------------------------------
// Colour-ordered Berends-Giele recursion for one event and one helicity.
// ------------------------------------------------------------------------------------
struct Params { double mt, wt, alphas; };

template <class R> struct Event {
  int k;            // number of gluons
  R P[7][4];        // physical momenta, particle order
  R q[5][4];        // incoming momentum of gluon g (= p for g1,g2, -p for final gluons)
  Cx<R> eps[5][4];  // gluon wavefunction for this helicity
  Cx<R> ubar[4], v[4];
};

inline int gluon_particle(int g) { return g < 2 ? g : g + 2; }

template <class R> struct Recursion {
  const Event<R>& ev;
  R gs, mt, wt;
  int base;
  std::vector<Cx<R>> J;       // gluon currents J(seq)[4]
  std::vector<R> PJ;          // incoming momentum of seq
  std::vector<char> haveJ;
  std::vector<Cx<R>> Psi;     // Psibar(prefix)[4]
  std::vector<char> havePsi;

  Recursion(const Event<R>& e, R g, R m, R w) : ev(e), gs(g), mt(m), wt(w) {
    base = e.k + 1;
    int size = 1;
    for (int i = 0; i < e.k; ++i) size *= base;
    J.assign(4 * size, Cx<R>()); PJ.assign(4 * size, R(0.0)); haveJ.assign(size, 0);
    Psi.assign(4 * size, Cx<R>()); havePsi.assign(size, 0);
  }
  int code(const int* seq, int len) const {
    int c = 0, w = 1;
    for (int i = 0; i < len; ++i) { c += (seq[i] + 1) * w; w *= base; }
    return c;
  }

  // J(seq): off-shell gluon current of the ordered gluons seq[0..len), including its
  // propagator; its momentum P is the sum of the incoming gluon momenta.
  const Cx<R>* current(const int* seq, int len, const R** Pout) {
    int c = code(seq, len);
    if (haveJ[c]) { *Pout = &PJ[4 * c]; return &J[4 * c]; }
    Cx<R>* out = &J[4 * c];
    R* P = &PJ[4 * c];
    if (len == 1) {
      for (int m = 0; m < 4; ++m) { out[m] = ev.eps[seq[0]][m]; P[m] = ev.q[seq[0]][m]; }
    } else {
      for (int m = 0; m < 4; ++m) P[m] = R(0.0);
      for (int i = 0; i < len; ++i)
        for (int m = 0; m < 4; ++m) P[m] = P[m] + ev.q[seq[i]][m];
      Cx<R> acc[4];
      // three-gluon vertex, every split seq = (L, R):
      // V3 = (JL.JR)(PL - PR) + (JL.(PL + 2 PR)) JR - (JR.(2 PL + PR)) JL, weight g
      for (int s = 1; s < len; ++s) {
        const R *PL, *PR;
        const Cx<R>* JL = current(seq, s, &PL);
        const Cx<R>* JR = current(seq + s, len - s, &PR);
        Cx<R> jj = dot_cc(JL, JR);
        R a1[4], a2[4], d[4];
        for (int m = 0; m < 4; ++m) { d[m] = PL[m] - PR[m]; a1[m] = PL[m] + R(2.0) * PR[m]; a2[m] = R(2.0) * PL[m] + PR[m]; }
        Cx<R> cL = dot_cr(JL, a1), cR = dot_cr(JR, a2);
        for (int m = 0; m < 4; ++m) {
          Cx<R> t = scale(d[m], jj) + cL * JR[m] - cR * JL[m];
          acc[m] = acc[m] + scale(gs, t);
        }
      }
      // four-gluon vertex, every split seq = (A, B, C):
      // V4 = (JA.JB) JC + (JB.JC) JA - 2 (JA.JC) JB, weight g^2
      for (int s1 = 1; s1 < len; ++s1) {
        for (int s2 = s1 + 1; s2 < len; ++s2) {
          const R *PA, *PB, *PC;
          const Cx<R>* JA = current(seq, s1, &PA);
          const Cx<R>* JB = current(seq + s1, s2 - s1, &PB);
          const Cx<R>* JC = current(seq + s2, len - s2, &PC);
          Cx<R> ab = dot_cc(JA, JB), bc = dot_cc(JB, JC), ac = dot_cc(JA, JC);
          for (int m = 0; m < 4; ++m) {
            Cx<R> t = ab * JC[m] + bc * JA[m] - scale(R(2.0), ac * JB[m]);
            acc[m] = acc[m] + scale(gs * gs, t);
          }
        }
      }
      // gluon propagator -i g^{mu nu}/P^2 times the vertex factor (-i) gives -1/P^2
      R f = R(-1.0) / dot_rr(P, P);
      for (int m = 0; m < 4; ++m) out[m] = scale(f, acc[m]);
    }
    haveJ[c] = 1;
    *Pout = P;
    return out;
  }

  // Psibar(prefix): ubar(p_t) with the ordered gluons prefix[0..len) attached along the
  // quark line, ending in the quark propagator S(Q) = i(Qslash + m)/(Q^2 - m^2 + i m w),
  // Q = p_t - P(prefix) flowing along the fermion arrow.
  const Cx<R>* psibar(const int* prefix, int len) {
    if (len == 0) return ev.ubar;
    int c = code(prefix, len);
    if (havePsi[c]) return &Psi[4 * c];
    Cx<R> acc[4];
    for (int j = 0; j < len; ++j) {
      const Cx<R>* left = psibar(prefix, j);
      const R* PJc;
      const Cx<R>* Jc = current(prefix + j, len - j, &PJc);
      Cx<R> t[4];
      row_gamma(left, Jc, t);
      // vertex i g gamma^mu
      for (int m = 0; m < 4; ++m) acc[m] = acc[m] + times_i(scale(gs, t[m]));
    }
    R Q[4];
    for (int m = 0; m < 4; ++m) Q[m] = ev.P[2][m];
    for (int i = 0; i < len; ++i)
      for (int m = 0; m < 4; ++m) Q[m] = Q[m] - ev.q[prefix[i]][m];
    Cx<R> num[4];
    row_qslash_plus_m(acc, Q, mt, num);
    // i / (Q^2 - m^2 + i m w)
    R dre = dot_rr(Q, Q) - mt * mt, dim = mt * wt;
    R nrm = R(1.0) / (dre * dre + dim * dim);
    Cx<R> prop(dim * nrm, dre * nrm);   // i (dre - i dim)/(dre^2+dim^2)
    Cx<R>* out = &Psi[4 * c];
    for (int m = 0; m < 4; ++m) out[m] = num[m] * prop;
    havePsi[c] = 1;
    return out;
  }

  // A(sigma) = sum_j Psibar(sigma_1..sigma_j) (i g gamma.J(sigma_{j+1}..sigma_k)) v(p_tbar)
  Cx<R> amplitude(const int* sigma) {
    int k = ev.k;
    Cx<R> A;
    for (int j = 0; j < k; ++j) {
      const Cx<R>* left = psibar(sigma, j);
      const R* PJc;
      const Cx<R>* Jc = current(sigma + j, k - j, &PJc);
      Cx<R> t[4];
      row_gamma(left, Jc, t);
      Cx<R> s = t[0] * ev.v[0] + t[1] * ev.v[1] + t[2] * ev.v[2] + t[3] * ev.v[3];
      A = A + times_i(scale(gs, s));
    }
    return A;
  }
};

// All permutations of 0..k-1 in lexicographic order.
std::vector<std::vector<int>> permutations(int k) {
  std::vector<int> p(k);
  for (int i = 0; i < k; ++i) p[i] = i;
  std::vector<std::vector<int>> out;
  do { out.push_back(p); } while (std::next_permutation(p.begin(), p.end()));
  return out;
}

// Load an event for helicity h.  gauge_gluon >= 0 replaces that gluon's polarisation by
// its momentum / E (gauge-invariance probe).
template <class R> void load_event(int k, const double* mom, int h, const Params& prm, int gauge_gluon, Event<R>& ev) {
  int npar = k + 2;
  ev.k = k;
  for (int i = 0; i < npar; ++i)
    for (int m = 0; m < 4; ++m) ev.P[i][m] = R(mom[4 * i + m]);
  auto lam = [&](int i) { return ((h >> (npar - 1 - i)) & 1) ? +1 : -1; };
  R mt(prm.mt);
  wf_ubar(ev.P[2], mt, lam(2), ev.ubar);
  wf_v(ev.P[3], mt, lam(3), ev.v);
  for (int g = 0; g < k; ++g) {
    int i = gluon_particle(g);
    bool incoming = g < 2;
    for (int m = 0; m < 4; ++m) ev.q[g][m] = incoming ? ev.P[i][m] : -ev.P[i][m];
    wf_eps(ev.P[i], lam(i), ev.eps[g]);
    if (!incoming)
      for (int m = 0; m < 4; ++m) ev.eps[g][m] = conj(ev.eps[g][m]);
    if (g == gauge_gluon) {
      R invE = R(1.0) / ev.P[i][0];
      for (int m = 0; m < 4; ++m) ev.eps[g][m] = Cx<R>(ev.P[i][m] * invE, R(0.0));
    }
  }
}

// Jamps of one event and helicity.
template <class R> void jamps_for(int k, const double* mom, int h, const Params& prm, int gauge_gluon,
                                  const std::vector<std::vector<int>>& perms, std::vector<Cx<R>>& A) {
  Event<R> ev;
  load_event<R>(k, mom, h, prm, gauge_gluon, ev);
  R gs = sqrt(R(4.0 * 3.14159265358979323846) * R(prm.alphas));
  Recursion<R> rec(ev, gs, R(prm.mt), R(prm.wt));
  A.resize(perms.size());
  for (size_t s = 0; s < perms.size(); ++s) A[s] = rec.amplitude(perms[s].data());
}

// sum_{sigma,tau} C(sigma,tau) Re(A_sigma A_tau^*), C real symmetric.
template <class R> R colour_sum(const std::vector<Cx<R>>& A, const double* colour) {
  int n = (int)A.size();
  R tot(0.0);
  for (int s = 0; s < n; ++s) {
    R rowre(0.0), rowim(0.0);
    for (int t = 0; t < n; ++t) {
      R c(colour[s * n + t]);
      rowre = rowre + c * A[t].re;
      rowim = rowim + c * A[t].im;
    }
    tot = tot + A[s].re * rowre + A[s].im * rowim;
  }
  return tot;
}

int nfact(int n) { int f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

}  // namespace

// =====================================================================================
// C entry points (ctypes).
// =====================================================================================
extern "C" {

void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

void orc_uniforms(uint64_t seed, uint64_t e, uint32_t j, double* u) { event_uniforms(seed, e, j, u); }

int orc_rambo(int n, const double* masses, const double* u, double sqrts, double* p, double* wgt) {
  return rambo(n, masses, u, sqrts, p, wgt);
}

// One event of g g -> t tbar + ng g: momenta mom[npar][4] (particle order g1 g2 t tbar g3..),
// final-state particle j of RAMBO draws its uniforms from counter {e, j}.
int orc_event(int ng, uint64_t seed, uint64_t e, double sqrts, double mt, double* mom, double* wgt) {
  int n = 2 + ng;
  double masses[5] = {mt, mt, 0, 0, 0};
  double u[20], p[20];
  for (int j = 0; j < n; ++j) event_uniforms(seed, e, (uint32_t)j, u + 4 * j);
  int st = rambo(n, masses, u, sqrts, p, wgt);
  double h = 0.5 * sqrts;
  double in[8] = {h, 0, 0, h, h, 0, 0, -h};
  std::memcpy(mom, in, sizeof(in));
  std::memcpy(mom + 8, p, sizeof(double) * 4 * n);
  return st;
}

int orc_events(int ng, uint64_t seed, int64_t e0, int64_t nevt, double sqrts, double mt, double* mom, double* wgt,
               int* status) {
  int npar = 4 + ng, bad = 0;
  for (int64_t i = 0; i < nevt; ++i) {
    double w;
    int st = orc_event(ng, seed, (uint64_t)(e0 + i), sqrts, mt, mom + 4 * npar * i, &w);
    if (wgt) wgt[i] = w;
    if (status) status[i] = st;
    if (st) bad++;
  }
  return bad;
}

// Per-helicity colour-summed |M_h|^2 (no averaging) for one event; optional jamps[nhel][ncol][2].
void orc_me_hel(int ng, const double* mom, const double* colour, double mt, double wt, double alphas, int gauge_gluon,
                double* mhel, double* jamps) {
  int k = ng + 2, npar = ng + 4, nhel = 1 << npar;
  Params prm = {mt, wt, alphas};
  auto perms = permutations(k);
  int ncol = (int)perms.size();
  std::vector<Cx<double>> A;
  for (int h = 0; h < nhel; ++h) {
    jamps_for<double>(k, mom, h, prm, gauge_gluon, perms, A);
    mhel[h] = colour_sum(A, colour);
    if (jamps)
      for (int s = 0; s < ncol; ++s) {
        jamps[2 * (h * ncol + s)] = A[s].re;
        jamps[2 * (h * ncol + s) + 1] = A[s].im;
      }
  }
}

// Helicity- and colour-summed |M|^2 averaged over initial helicities and colours (1/256)
// and divided by ng! for identical final-state gluons, summing the helicities whose bit
// is set in mask (bit h of word h/32).  Events are split over nthreads std::threads.
void orc_me_batch(int ng, int64_t nevt, const double* mom, const double* colour, double mt, double wt, double alphas,
                  const uint32_t* mask, double* me, int nthreads) {
  int k = ng + 2, npar = ng + 4, nhel = 1 << npar;
  Params prm = {mt, wt, alphas};
  auto perms = permutations(k);
  double norm = 1.0 / (256.0 * nfact(ng));
  auto work = [&](int64_t lo, int64_t hi) {
    std::vector<Cx<double>> A;
    for (int64_t e = lo; e < hi; ++e) {
      const double* p = mom + 4 * npar * e;
      double tot = 0;
      for (int h = 0; h < nhel; ++h) {
        if (!((mask[h >> 5] >> (h & 31)) & 1u)) continue;
        jamps_for<double>(k, p, h, prm, -1, perms, A);
        tot += colour_sum(A, colour);
      }
      me[e] = tot * norm;
    }
  };
  if (nthreads <= 1) { work(0, nevt); return; }
  std::vector<std::thread> th;
  int64_t chunk = (nevt + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    int64_t lo = t * chunk, hi = std::min<int64_t>(nevt, lo + chunk);
    if (lo < hi) th.emplace_back(work, lo, hi);
  }
  for (auto& x : th) x.join();
}

// Operation counts of one event's matrix element over the helicities in mask:
// counts = {add, mul, div, sqrt} for the amplitudes (wavefunctions, currents, jamps)
// followed by {add, mul, div, sqrt} for the colour sums.
void orc_flops(int ng, const double* mom, const double* colour, double mt, double wt, double alphas,
               const uint32_t* mask, unsigned long long* counts) {
  int k = ng + 2, npar = ng + 4, nhel = 1 << npar;
  Params prm = {mt, wt, alphas};
  auto perms = permutations(k);
  Counter amp = {0, 0, 0, 0}, col = {0, 0, 0, 0};
  std::vector<Cx<Cd>> A;
  for (int h = 0; h < nhel; ++h) {
    if (!((mask[h >> 5] >> (h & 31)) & 1u)) continue;
    tl_count = Counter{0, 0, 0, 0};
    jamps_for<Cd>(k, mom, h, prm, -1, perms, A);
    Counter a = tl_count;
    tl_count = Counter{0, 0, 0, 0};
    (void)colour_sum(A, colour);
    Counter c = tl_count;
    amp.add += a.add; amp.mul += a.mul; amp.div += a.div; amp.sqrt += a.sqrt;
    col.add += c.add; col.mul += c.mul; col.div += c.div; col.sqrt += c.sqrt;
  }
  counts[0] = amp.add; counts[1] = amp.mul; counts[2] = amp.div; counts[3] = amp.sqrt;
  counts[4] = col.add; counts[5] = col.mul; counts[6] = col.div; counts[7] = col.sqrt;
}

// Helicity filter over warm-up events: good(h) <=> max_e |M_h|^2 / sum_h' |M_h'|^2 > tau.
// maxratio[h] receives the maximum ratio; mask has ceil(nhel/32) words.  Events are split
// over nthreads std::threads (the maximum does not depend on the split).
void orc_hel_mask(int ng, int64_t nevt, const double* mom, const double* colour, double mt, double wt, double alphas,
                  double tau, uint32_t* mask, double* maxratio, int nthreads) {
  int npar = ng + 4, nhel = 1 << npar;
  if (nthreads < 1) nthreads = 1;
  std::vector<std::vector<double>> part(nthreads, std::vector<double>(nhel, 0.0));
  auto work = [&](int t) {
    std::vector<double> mh(nhel);
    for (int64_t e = t; e < nevt; e += nthreads) {
      orc_me_hel(ng, mom + 4 * npar * e, colour, mt, wt, alphas, -1, mh.data(), nullptr);
      double tot = 0;
      for (int h = 0; h < nhel; ++h) tot += mh[h];
      for (int h = 0; h < nhel; ++h) part[t][h] = std::max(part[t][h], mh[h] / tot);
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) th.emplace_back(work, t);
  for (auto& x : th) x.join();
  for (int h = 0; h < nhel; ++h) {
    maxratio[h] = 0;
    for (int t = 0; t < nthreads; ++t) maxratio[h] = std::max(maxratio[h], part[t][h]);
  }
  int nw = (nhel + 31) / 32;
  for (int w = 0; w < nw; ++w) mask[w] = 0;
  for (int h = 0; h < nhel; ++h)
    if (maxratio[h] > tau) mask[h >> 5] |= 1u << (h & 31);
}

}  // extern "C"
