"""Brute-force colour-dressed tree amplitudes with explicit SU(3) matrices -- TEST INFRASTRUCTURE ONLY.

An independent second calculation of sum_colours |M_h|^2 for g g -> t tbar + n_g g, used to
pin the colour decomposition, the colour matrix and the colour-ordered rules of me_oracle.cpp.
It uses the standard (not colour-ordered) Feynman-gauge QCD Feynman rules with explicit
Gell-Mann matrices T^a = lambda^a / 2 and structure constants f^{abc} = -2i Tr([T^a,T^b] T^c):

    quark-gluon vertex   i g gamma^mu (T^a)_{ij}
    three-gluon vertex   g f^{abc} [g^{mu nu}(k1-k2)^rho + g^{nu rho}(k2-k3)^mu + g^{rho mu}(k3-k1)^nu]
    four-gluon vertex    -i g^2 [f^{abe} f^{cde}(g^{mu rho} g^{nu sigma} - g^{mu sigma} g^{nu rho})
                                + f^{ace} f^{bde}(g^{mu nu} g^{rho sigma} - g^{mu sigma} g^{nu rho})
                                + f^{ade} f^{bce}(g^{mu nu} g^{rho sigma} - g^{mu rho} g^{nu sigma})]
    gluon propagator     -i g_{mu nu} delta^{ab} / k^2
    quark propagator     i (pslash + m) / (p^2 - m^2)

(Peskin-Schroeder Sec. 16.1 conventions; all three-gluon momenta incoming).  Every tree
diagram is summed once by a Berends-Giele recursion over UNORDERED gluon subsets, each
current carrying the explicit adjoint indices of its external gluons, and |M|^2 is summed
over every colour index by brute force.  The wavefunctions are written here from their
angle-based definitions (Murayama-Watanabe-Hagiwara HELAS conventions), independently of
me_oracle.cpp.  Also: a diagram-counting version of the same recursion.

Cost grows as 8^k; meant for k <= 4 gluons and a handful of events.
"""
import itertools
import math
from functools import lru_cache

import numpy as np

METRIC = np.diag([1.0, -1.0, -1.0, -1.0])


# ----------------------------------------------------------------------------------------
# SU(3) generators and structure constants
# ----------------------------------------------------------------------------------------
def gell_mann():
    l = np.zeros((8, 3, 3), dtype=complex)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j
    l[1][1, 0] = 1j
    l[2][0, 0] = 1
    l[2][1, 1] = -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j
    l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j
    l[6][2, 1] = 1j
    l[7][0, 0] = l[7][1, 1] = 1 / math.sqrt(3)
    l[7][2, 2] = -2 / math.sqrt(3)
    return l


T = gell_mann() / 2.0


def structure_constants():
    comm = np.einsum("aij,bjk->abik", T, T) - np.einsum("bij,ajk->abik", T, T)
    f = -2j * np.einsum("abij,cji->abc", comm, T)
    assert np.abs(f.imag).max() < 1e-14
    return f.real


F = structure_constants()

# chiral-representation gamma matrices (upper index), gamma^mu = [[0, sigma^mu], [sigmabar^mu, 0]]
_S = [np.eye(2, dtype=complex), np.array([[0, 1], [1, 0]], dtype=complex),
      np.array([[0, -1j], [1j, 0]], dtype=complex), np.array([[1, 0], [0, -1]], dtype=complex)]
GAMMA = np.zeros((4, 4, 4), dtype=complex)
for _mu in range(4):
    sig = _S[_mu]
    sbar = _S[0] if _mu == 0 else -_S[_mu]
    GAMMA[_mu][:2, 2:] = sig
    GAMMA[_mu][2:, :2] = sbar
GAMMA0 = GAMMA[0]


# ----------------------------------------------------------------------------------------
# wavefunctions from angles
# ----------------------------------------------------------------------------------------
def _angles(p3):
    pp = np.linalg.norm(p3)
    theta = math.acos(max(-1.0, min(1.0, p3[2] / pp)))
    phi = math.atan2(p3[1], p3[0]) if (p3[0] != 0 or p3[1] != 0) else 0.0
    return pp, theta, phi


def chi(p3, lam):
    """Two-component helicity eigenspinor: chi_+ = (cos t/2, e^{i phi} sin t/2), chi_- = (-e^{-i phi} sin t/2, cos t/2)."""
    _, th, ph = _angles(p3)
    if lam > 0:
        return np.array([math.cos(th / 2), np.exp(1j * ph) * math.sin(th / 2)])
    return np.array([-np.exp(-1j * ph) * math.sin(th / 2), math.cos(th / 2)])


def spinor_u(p, m, lam):
    pp = np.linalg.norm(p[1:])
    E = p[0]
    c = chi(p[1:], lam)
    return np.concatenate([math.sqrt(max(E - lam * pp, 0.0)) * c, math.sqrt(max(E + lam * pp, 0.0)) * c])


def spinor_v(p, m, lam):
    """Outgoing antifermion of physical helicity lam."""
    pp = np.linalg.norm(p[1:])
    E = p[0]
    c = chi(p[1:], -lam)
    return np.concatenate([-lam * math.sqrt(max(E + lam * pp, 0.0)) * c, lam * math.sqrt(max(E - lam * pp, 0.0)) * c])


def spinor_ubar(p, m, lam):
    u = spinor_u(p, m, lam)
    return u.conj() @ GAMMA0


def polarisation(k, lam):
    """epsilon^mu(k, lam) = (0, (-lam e_theta - i e_phi)/sqrt 2)."""
    _, th, ph = _angles(k[1:])
    e_th = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
    e_ph = np.array([-math.sin(ph), math.cos(ph), 0.0])
    e = np.zeros(4, dtype=complex)
    e[1:] = (-lam * e_th - 1j * e_ph) / math.sqrt(2)
    return e


# ----------------------------------------------------------------------------------------
# colour-dressed recursion
# ----------------------------------------------------------------------------------------
def _v3_tensor(k1, k2, k3):
    """V^{mu nu rho}(k1,k2,k3) with upper indices."""
    g = np.linalg.inv(METRIC)  # g^{mu nu}
    V = (np.einsum("mn,r->mnr", g, k1 - k2) + np.einsum("nr,m->mnr", g, k2 - k3)
         + np.einsum("rm,n->mnr", g, k3 - k1))
    return V


def _lower(J):
    return J * np.array([1.0, -1.0, -1.0, -1.0])


def _subsets(mask):
    """Nonempty proper subsets of the bitmask."""
    sub = (mask - 1) & mask
    while sub:
        yield sub
        sub = (sub - 1) & mask


def helicity_me(ng, p, hel, mt, alphas, want_amplitude=False):
    """sum over all colours of |M_h|^2 for event p[npar][4] and helicity index hel."""
    k = ng + 2
    npar = ng + 4
    gs = math.sqrt(4 * math.pi * alphas)
    lam = [1 if (hel >> (npar - 1 - i)) & 1 else -1 for i in range(npar)]
    part = [g if g < 2 else g + 2 for g in range(k)]
    q = [p[part[g]] if g < 2 else -p[part[g]] for g in range(k)]
    eps = []
    for g in range(k):
        e = polarisation(p[part[g]], lam[part[g]])
        eps.append(e if g < 2 else e.conj())

    def shape_for(mask, tail):
        return tuple(8 if (mask >> g) & 1 else 1 for g in range(k)) + tail

    J = {}
    Pm = {}
    full = (1 << k) - 1
    for mask in sorted(range(1, full + 1), key=lambda m: bin(m).count("1")):
        P = sum(q[g] for g in range(k) if (mask >> g) & 1)
        Pm[mask] = P
        if bin(mask).count("1") == 1:
            g = mask.bit_length() - 1
            arr = np.zeros(shape_for(mask, (8, 4)), dtype=complex)
            idx = [0] * k
            for a in range(8):
                idx[g] = a
                arr[tuple(idx) + (a,)] = eps[g]
            J[mask] = arr
            continue
        acc = np.zeros(shape_for(mask, (8, 4)), dtype=complex)
        # three-gluon vertex: unordered pairs {S1, S2}
        for s1 in _subsets(mask):
            s2 = mask ^ s1
            if s1 > s2:
                continue
            V = _v3_tensor(Pm[s1], Pm[s2], -P)  # legs (S1: nu), (S2: rho), (off-shell: mu) -> order (nu, rho, mu)
            # contract J1_nu J2_rho V^{nu rho mu}
            t = np.einsum("...bn,...cr,nrm->...bcm", _lower(J[s1]), _lower(J[s2]), V, optimize=True)
            acc = acc + gs * np.einsum("...bcm,bce->...em", t, F)
        # four-gluon vertex: unordered triples {S1, S2, S3}
        for s1 in _subsets(mask):
            rest = mask ^ s1
            for s2 in _subsets(rest) if rest else []:
                s3 = rest ^ s2
                if not (s1 < s2 < s3):
                    continue
                A, B, C = _lower(J[s1]), _lower(J[s2]), _lower(J[s3])
                # legs: (b, nu) = S1, (c, rho) = S2, (d, sig) = S3, (e, mu) = off-shell, mu raised at the end
                # dot products J_i . J_j = (J_i)_mu (J_j)^mu
                ab = np.einsum("...bn,...cn->...bc", A, J[s2])
                ac = np.einsum("...bn,...dn->...bd", A, J[s3])
                bc = np.einsum("...cn,...dn->...cd", B, J[s3])
                # vertex with the off-shell leg (e, mu) as the FIRST leg (a, mu) of the rule:
                # f^{e b x} f^{c d x}(g^{mu rho} g^{nu sig} - g^{mu sig} g^{nu rho})
                # + f^{e c x} f^{b d x}(g^{mu nu} g^{rho sig} - g^{mu sig} g^{nu rho})
                # + f^{e d x} f^{b c x}(g^{mu nu} g^{rho sig} - g^{mu rho} g^{nu sig})
                ff1 = np.einsum("ebx,cdx->ebcd", F, F)
                ff2 = np.einsum("ecx,bdx->ebcd", F, F)
                ff3 = np.einsum("edx,bcx->ebcd", F, F)
                Ju, Ku, Lu = J[s1], J[s2], J[s3]
                # term1: (J2^mu)(J1.J3) - (J3^mu)(J1.J2)
                t1 = (np.einsum("ebcd,...bd,...cm->...em", ff1, ac, Ku, optimize=True)
                      - np.einsum("ebcd,...bc,...dm->...em", ff1, ab, Lu, optimize=True))
                # term2: (J1^mu)(J2.J3) - (J3^mu)(J1.J2)
                t2 = (np.einsum("ebcd,...cd,...bm->...em", ff2, bc, Ju, optimize=True)
                      - np.einsum("ebcd,...bc,...dm->...em", ff2, ab, Lu, optimize=True))
                # term3: (J1^mu)(J2.J3) - (J2^mu)(J1.J3)
                t3 = (np.einsum("ebcd,...cd,...bm->...em", ff3, bc, Ju, optimize=True)
                      - np.einsum("ebcd,...bd,...cm->...em", ff3, ac, Ku, optimize=True))
                acc = acc + (-1j * gs * gs) * (t1 + t2 + t3)
        # gluon propagator -i g/P^2 (index raised: the accumulated vertex has an upper index)
        J[mask] = (-1j / (P @ METRIC @ P)) * acc

    # fermion line: Psibar(S)[..., i_t, c, s]
    ubar = spinor_ubar(p[2], mt, lam[2])
    v = spinor_v(p[3], mt, lam[3])
    slash = lambda Jv: np.einsum("...m,mst->...st", _lower(Jv), GAMMA)  # gamma^mu J_mu
    Psi = {}
    base = np.zeros(shape_for(0, (3, 3, 4)), dtype=complex)
    for i in range(3):
        base[(0,) * k + (i, i)] = ubar
    Psi[0] = base
    for mask in sorted(range(1, full), key=lambda m: bin(m).count("1")):
        acc = np.zeros(shape_for(mask, (3, 3, 4)), dtype=complex)
        for t in itertools.chain([mask], _subsets(mask)):
            left = Psi[mask ^ t]
            G = slash(J[t])                        # [..., e, s, s']
            # left[..., i, c, s] (i g gamma T^e)_{s s'} (T^e)_{c c'} J^e
            acc = acc + 1j * gs * np.einsum("...ics,...est,ecd->...idt", left, G, T, optimize=True)
        Q = p[2] - Pm[mask]
        num = (np.einsum("m,mst->st", METRIC @ Q, GAMMA) + mt * np.eye(4))
        Psi[mask] = np.einsum("...ics,st->...ict", acc, num) * (1j / (Q @ METRIC @ Q - mt * mt))
    M = np.zeros(shape_for(full, (3, 3)), dtype=complex)
    for t in itertools.chain([full], _subsets(full)):
        left = Psi[full ^ t]
        G = slash(J[t])
        M = M + 1j * gs * np.einsum("...ics,...est,ecj,t->...ij", left, G, T, v, optimize=True)
    val = float(np.sum(np.abs(M) ** 2))
    if want_amplitude:
        return val, M
    return val


def me_hel(ng, p, mt, alphas):
    return np.array([helicity_me(ng, p, h, mt, alphas) for h in range(1 << (ng + 4))])


# ----------------------------------------------------------------------------------------
# diagram counting: the same recursion over unordered subsets with every vertex worth 1
# ----------------------------------------------------------------------------------------
def count_diagrams(k):
    @lru_cache(maxsize=None)
    def gluon(mask):
        if bin(mask).count("1") == 1:
            return 1
        n = 0
        for s1 in _subsets(mask):
            s2 = mask ^ s1
            if s1 < s2:
                n += gluon(s1) * gluon(s2)
        for s1 in _subsets(mask):
            rest = mask ^ s1
            for s2 in (_subsets(rest) if rest else []):
                s3 = rest ^ s2
                if s1 < s2 < s3:
                    n += gluon(s1) * gluon(s2) * gluon(s3)
        return n

    @lru_cache(maxsize=None)
    def quark(mask):
        if mask == 0:
            return 1
        return sum(quark(mask ^ t) * gluon(t) for t in itertools.chain([mask], _subsets(mask)))

    full = (1 << k) - 1
    return sum(quark(full ^ t) * gluon(t) for t in itertools.chain([full], _subsets(full)))
