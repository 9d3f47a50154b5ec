"""Single-diagram-enhancement channel weights -- TEST INFRASTRUCTURE ONLY.

The paper (arXiv 2210.11122, Sec. 2) lists MadEvent's single-diagram-enhancement algorithm among the
features its GPU matrix-element engine gained.  For phase-space integration channel d (a Feynman
diagram) the event weight is multiplied by

    w_d = sum_h |A_d(h)|^2 / sum_d' sum_h |A_d'(h)|^2,

A_d the amplitude of diagram d alone with its colour factor stripped, summed over the good helicities.
Reading (the paper gives no definition): the channels are the tree diagrams built from three-point
vertices only -- a diagram with a four-gluon vertex has no propagator structure of its own -- and the
colour-stripped vertices are the Feynman-gauge ones with the couplings and phases dropped (every channel
has n_g + 2 vertices, so g and the phases are common to all and cancel in w_d):
    quark-gluon    gamma^mu
    three-gluon    g^{mu nu}(k1 - k2)^rho + g^{nu rho}(k2 - k3)^mu + g^{rho mu}(k3 - k1)^nu  (momenta incoming)
    propagators    gluon 1/P^2, top (Qslash + m)/(Q^2 - m^2).
A diagram is the ordered list of gluon trees attached along the quark line from the top (ubar) to the
antitop (v); each tree is a binary tree over a subset of the gluons, the subsets partitioning them.

Written directly from those rules with the 4x4 gamma matrices of fullcolour.py and wavefunctions of its
own (the HELAS helicity states in the chiral basis, from the momentum components: cos(theta/2) and
sin(theta/2) as square roots of (|p| +- pz) / 2|p|, the form of |p| + pz without cancellation for pz < 0,
so every component keeps full FP64 precision near the beam axis, where angles from acos do not),
independently of me_oracle.cpp.  Channel keys: a gluon tree is its leaf label (1-based
gluon index: 1, 2 incoming, 3.. outgoing) or "(A,B)" with the child holding the smaller label first;
a diagram joins its trees with "|" in quark-line order.
"""
import itertools
import math

import numpy as np

from . import fullcolour as fc


def trees(labels, four=False):
    """Every tree over the sorted tuple of gluon labels: a leaf, or a node joining two (or, with four, also
    three) subtrees over a partition of the labels; each unordered partition once."""
    if len(labels) == 1:
        return [labels[0]]
    out = []
    first, rest = labels[0], labels[1:]
    for r in range(len(rest)):                     # the part holding `first` takes r of the rest
        for extra in itertools.combinations(rest, r):
            a = (first,) + extra
            b = tuple(x for x in rest if x not in extra)
            for ta in trees(a, four):
                for tb in trees(b, four):
                    out.append((ta, tb))
    if four and len(labels) >= 3:
        for r in range(len(rest) - 1):             # three parts: `first`'s, then the smallest remaining's
            for extra in itertools.combinations(rest, r):
                a = (first,) + extra
                left = tuple(x for x in rest if x not in extra)
                f2, rest2 = left[0], left[1:]
                for r2 in range(len(rest2)):
                    for extra2 in itertools.combinations(rest2, r2):
                        b = (f2,) + extra2
                        c = tuple(x for x in rest2 if x not in extra2)
                        for ta in trees(a, four):
                            for tb in trees(b, four):
                                for tc in trees(c, four):
                                    out.append((ta, tb, tc))
    return out


def diagrams(ng, four=False):
    """Every diagram: ordered lists of trees along the quark line, their label sets partitioning the gluons."""
    def seq(rem):
        if not rem:
            return [[]]
        out = []
        for r in range(1, len(rem) + 1):
            for s in itertools.combinations(rem, r):
                rest = tuple(x for x in rem if x not in s)
                for t in trees(s, four):
                    for tail in seq(rest):
                        out.append([t] + tail)
        return out
    return seq(tuple(range(ng + 2)))


def tree_key(t):
    if isinstance(t, int):
        return str(t + 1)
    return "(" + ",".join(tree_key(c) for c in t) + ")"


def key(d):
    return "|".join(tree_key(t) for t in d)


def _slash(J):
    """gamma^mu J_mu for a contravariant J."""
    return fc.GAMMA[0] * J[0] - fc.GAMMA[1] * J[1] - fc.GAMMA[2] * J[2] - fc.GAMMA[3] * J[3]


def _dot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def _v3(jl, pl, jr, pr):
    """Three-gluon vertex contracted with the currents of momenta pl, pr (incoming); contravariant vector."""
    return _dot(jl, jr) * (pl - pr) + _dot(jl, pl + 2 * pr) * jr - _dot(jr, 2 * pl + pr) * jl


def _chi(p3, lam):
    """Two-component helicity eigenspinor (sigma.p) chi = lam |p| chi: chi_+ = (cos t/2, e^{i phi} sin t/2),
    chi_- = (-e^{-i phi} sin t/2, cos t/2), from the components (the theta -> pi limit at phi = 0 on -z)."""
    px, py, pz = p3
    pt2 = px * px + py * py
    pp = math.sqrt(pt2 + pz * pz)
    ppz = pp + pz if pz >= 0 else pt2 / (pp - pz)          # |p| + pz
    if ppz <= 0:
        return np.array([0, 1], dtype=complex) if lam > 0 else np.array([-1, 0], dtype=complex)
    n = 1 / math.sqrt(2 * pp * ppz)
    c, sp = ppz * n, complex(px, py) * n                   # cos t/2, e^{i phi} sin t/2
    return np.array([c, sp]) if lam > 0 else np.array([-sp.conjugate(), c])


def _ubar(p, m, lam):
    """ubar = u^dagger gamma^0, u = (sqrt(E - lam|p|) chi_lam ; sqrt(E + lam|p|) chi_lam)."""
    pp = math.sqrt(p[1] ** 2 + p[2] ** 2 + p[3] ** 2)
    wp = math.sqrt(p[0] + pp)
    wm = m / wp if m > 0 else 0.0                          # sqrt(E - |p|) = m / sqrt(E + |p|)
    c = _chi(p[1:], lam)
    u = np.concatenate([(wm if lam > 0 else wp) * c, (wp if lam > 0 else wm) * c])
    return u.conj() @ fc.GAMMA0


def _v(p, m, lam):
    """Outgoing antifermion of physical helicity lam: (-lam sqrt(E + lam|p|) chi_-lam ; lam sqrt(E - lam|p|) chi_-lam)."""
    pp = math.sqrt(p[1] ** 2 + p[2] ** 2 + p[3] ** 2)
    wp = math.sqrt(p[0] + pp)
    wm = m / wp if m > 0 else 0.0
    c = _chi(p[1:], -lam)
    return np.concatenate([(-wp if lam > 0 else wm) * c, (wm if lam > 0 else -wp) * c])


def _eps(k, lam):
    """epsilon(k, lam) = (0, (-lam e_theta - i e_phi)/sqrt 2) from the components (phi = 0 on the z axis)."""
    kx, ky, kz = k[1], k[2], k[3]
    kt = math.sqrt(kx * kx + ky * ky)
    kk = math.sqrt(kt * kt + kz * kz)
    if kt > 0:
        e_th = np.array([kx * kz / (kk * kt), ky * kz / (kk * kt), -kt / kk])
        e_ph = np.array([-ky / kt, kx / kt, 0.0])
    else:
        e_th = np.array([1.0 if kz >= 0 else -1.0, 0.0, 0.0])
        e_ph = np.array([0.0, 1.0, 0.0])
    e = np.zeros(4, dtype=complex)
    e[1:] = (-lam * e_th - 1j * e_ph) / math.sqrt(2)
    return e


def externals(ng, p, hel, mt):
    npar = ng + 4
    lam = [1 if (hel >> (npar - 1 - i)) & 1 else -1 for i in range(npar)]
    part = [g if g < 2 else g + 2 for g in range(ng + 2)]
    q = [np.array(p[part[g]], dtype=float) if g < 2 else -np.array(p[part[g]], dtype=float) for g in range(ng + 2)]
    eps = []
    for g in range(ng + 2):
        e = _eps(np.array(p[part[g]], dtype=float), lam[part[g]])
        eps.append(e if g < 2 else e.conj())
    ub = _ubar(np.array(p[2], dtype=float), mt, lam[2])
    v = _v(np.array(p[3], dtype=float), mt, lam[3])
    return q, eps, ub, v


def amplitudes(ng, p, hel, mt=173.0, dias=None):
    """Colour-stripped amplitude of every channel (three-point vertices only) for one event and helicity."""
    dias = diagrams(ng) if dias is None else dias
    q, eps, ub, v = externals(ng, p, hel, mt)
    cache = {}

    def cur(t):
        if isinstance(t, int):
            return eps[t], q[t]
        k = tree_key(t)
        if k not in cache:
            jl, pl = cur(t[0])
            jr, pr = cur(t[1])
            P = pl + pr
            cache[k] = (_v3(jl, pl, jr, pr) / _dot(P, P), P)
        return cache[k]

    pt = np.array(p[2], dtype=float)
    out = np.zeros(len(dias), dtype=complex)
    for i, d in enumerate(dias):
        row = ub
        Q = pt.copy()
        for n, t in enumerate(d):
            J, P = cur(t)
            row = row @ _slash(J)
            Q = Q - P
            if n + 1 < len(d):
                row = row @ (_slash(Q.astype(complex)) + mt * np.eye(4)) / (_dot(Q, Q) - mt * mt)
        out[i] = row @ v
    return out


def weights(ng, p, mask, mt=173.0, dias=None):
    """w_d of every channel for one event: sum over the good helicities of |A_d|^2, normalised to 1."""
    dias = diagrams(ng) if dias is None else dias
    acc = np.zeros(len(dias))
    for h in range(1 << (ng + 4)):
        if (int(mask[h >> 5]) >> (h & 31)) & 1:
            a = amplitudes(ng, p, h, mt, dias)
            acc += a.real ** 2 + a.imag ** 2
    return acc / acc.sum()
