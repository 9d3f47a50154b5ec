"""Pins of the FP64 oracle against what the mathematics fixes (CPU only, no GPU).

Each test checks the oracle against something other than itself: a library routine, a
closed form, an exact identity, an invariance of the S-matrix, or an independent brute-force
calculation (oracle/fullcolour.py, written from the standard Feynman rules with explicit SU(3)
matrices).  The workflow pinned here is the paper's random numbers -> momenta -> matrix
element per event (arXiv 2210.11122, Sec. 1, Fig. 1; Sec. 2).
"""
import ctypes
import ctypes.util
import math
import os
from fractions import Fraction
from itertools import permutations

import numpy as np
import pytest

SQRTS, MT, AS = 1500.0, 173.0, 0.118


# ----------------------------------------------------------------------------------------
# Philox4x32-10
# ----------------------------------------------------------------------------------------
def _curand():
    cands = [ctypes.util.find_library("curand"), "/usr/local/cuda/lib64/libcurand.so", "libcurand.so.10"]
    for c in cands:
        if not c:
            continue
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 2**64 - 1])
def test_philox_matches_curand_host_generator(orc, seed):
    """cuRAND's host-side PHILOX4_32_10 generator (library code run on the CPU) emits, for seed s,
    word 4i+j = Philox4x32-10(counter (0, 0, i, 0), key (s_lo, s_hi))[j]."""
    L = _curand()
    if L is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert L.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4096
        out = np.zeros(n, dtype=np.uint32)
        assert L.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        L.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    ref = np.concatenate([orc.philox([0, 0, i, 0], key) for i in range(n // 4)])
    assert np.array_equal(out, ref)


def test_event_uniform_mapping(orc):
    """u = (x + 0.5) 2^-32 from counter {e_lo, e_hi, j, 0}, key {seed_lo, seed_hi}."""
    seed, e = 0xDEADBEEF12345678, (7 << 32) + 11
    for j in range(5):
        x = orc.philox([e & 0xFFFFFFFF, e >> 32, j, 0], [seed & 0xFFFFFFFF, seed >> 32])
        u = orc.uniforms(seed, e, j)
        assert np.array_equal(u, (x.astype(np.float64) + 0.5) * 2.0**-32)
        assert np.all((u > 0) & (u < 1))


# ----------------------------------------------------------------------------------------
# RAMBO
# ----------------------------------------------------------------------------------------
def mdot(a, b):
    return a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]


@pytest.mark.parametrize("ng", [0, 1, 2, 3])
def test_rambo_conservation_and_mass_shell(orc, ng):
    mom, w, st = orc.events(ng, 10 + ng, 2000)
    assert np.all(st == 0)
    fin = mom[:, 2:, :].sum(axis=1)
    assert np.max(np.abs(fin - np.array([SQRTS, 0, 0, 0]))) <= 1e-12 * SQRTS
    ini = mom[:, 0, :] + mom[:, 1, :]
    assert np.max(np.abs(ini - np.array([SQRTS, 0, 0, 0]))) == 0.0
    for i in (2, 3):
        m2 = mdot(mom[:, i], mom[:, i])
        assert np.max(np.abs(m2 / MT**2 - 1.0)) <= 1e-10
    for i in range(4, 4 + ng):
        m2 = mdot(mom[:, i], mom[:, i])
        assert np.max(np.abs(m2)) <= 1e-12 * SQRTS**2
    assert np.all(mom[:, 2:, 0] > 0)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_rambo_massless_weight_is_flat_volume(orc, n):
    """Massless n-body phase-space volume (2pi)^(4-3n) (pi/2)^(n-1) s^(n-2) / ((n-1)!(n-2)!)."""
    rng = np.random.default_rng(n)
    vol = (2 * math.pi) ** (4 - 3 * n) * (math.pi / 2) ** (n - 1) * SQRTS ** (2 * (n - 2)) / (
        math.factorial(n - 1) * math.factorial(n - 2))
    for _ in range(20):
        u = rng.uniform(0.01, 0.99, size=(n, 4))
        p, w, st = orc.rambo(np.zeros(n), u, SQRTS)
        assert st == 0
        assert abs(w / vol - 1) < 1e-13
        assert np.max(np.abs(mdot(p, p))) < 1e-10 * SQRTS**2


def test_rambo_two_body_massive_weight(orc):
    """Two-body phase space with equal masses: beta / (8 pi), beta = sqrt(1 - 4 m^2 / s)."""
    mom, w, st = orc.events(0, 3, 100)
    beta = math.sqrt(1 - 4 * MT**2 / SQRTS**2)
    assert np.max(np.abs(w / (beta / (8 * math.pi)) - 1)) < 1e-12


def test_rambo_three_body_massive_volume(orc):
    """Mean massive RAMBO weight = 3-body phase-space volume, computed independently as the Dalitz-plot
    area / (16 s (2pi)^3) (PDG kinematics), for t tbar g at sqrt(s) = 1500."""
    from scipy.integrate import quad
    s = SQRTS**2
    m1 = m2 = MT
    m3 = 0.0

    def m23_range(m12sq):
        # PDG: E2*, E3* in the (12) rest frame
        m12 = math.sqrt(m12sq)
        e2 = (m12sq - m1**2 + m2**2) / (2 * m12)
        e3 = (s - m12sq - m3**2) / (2 * m12)
        p2 = math.sqrt(max(e2**2 - m2**2, 0))
        p3 = math.sqrt(max(e3**2 - m3**2, 0))
        return (e2 + e3) ** 2 - (p2 + p3) ** 2, (e2 + e3) ** 2 - (p2 - p3) ** 2

    area, _ = quad(lambda x: m23_range(x)[1] - m23_range(x)[0], (m1 + m2) ** 2, (SQRTS - m3) ** 2,
                   epsabs=0, epsrel=1e-12, limit=200)
    vol = area / (16 * s * (2 * math.pi) ** 3)
    _, w, st = orc.events(1, 99, 200000)
    assert np.all(st == 0)
    mean, err = w.mean(), w.std() / math.sqrt(len(w))
    assert abs(mean - vol) < 5 * err
    assert err / vol < 3e-3


# ----------------------------------------------------------------------------------------
# matrix element: closed form, brute force, invariances
# ----------------------------------------------------------------------------------------
def test_ggtt_closed_form(orc):
    from oracle.closed_form import ggtt_me
    mom, _, _ = orc.events(0, 1, 512)
    me = orc.me_batch(0, mom)
    ref = ggtt_me(mom, MT, AS)
    # gauge cancellations between the three diagrams amplify rounding to ~1e-13 at worst
    assert np.max(np.abs(me / ref - 1)) < 1e-12
    assert np.median(np.abs(me / ref - 1)) < 1e-14


def test_ggtt_closed_form_massless_limit(orc):
    from oracle.closed_form import ggtt_me
    mom, _, st = orc.events(0, 2, 256, mt=0.0)
    assert np.all(st == 0)
    me = orc.me_batch(0, mom, mt=0.0)
    ref = ggtt_me(mom, 0.0, AS)
    # The closed form assumes exactly on-shell momenta; RAMBO's FP64 momenta are off shell by
    # ~1e-13 E^2, which near-collinear events (small 2 p1.p4) amplify to a few 1e-12.
    assert np.max(np.abs(me / ref - 1)) < 2e-11
    assert np.median(np.abs(me / ref - 1)) < 1e-14


@pytest.mark.parametrize("ng,nev,hels", [(0, 2, None), (1, 1, None), (2, 1, [0, 21, 42, 63])])
def test_full_colour_brute_force(orc, ng, nev, hels):
    """Colour-ordered recursion x exact colour matrix == explicit SU(3) sum over all Feynman diagrams."""
    from oracle import fullcolour as fc
    mom, _, _ = orc.events(ng, 40 + ng, nev)
    for e in range(nev):
        mh = orc.me_hel(ng, mom[e])
        hs = range(len(mh)) if hels is None else hels
        for h in hs:
            ref = fc.helicity_me(ng, mom[e], h, MT, AS)
            assert abs(mh[h] - ref) <= 1e-12 * mh.max()
            if ref > 1e-10 * mh.max():
                assert abs(mh[h] / ref - 1) < 1e-11


def _mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


@pytest.mark.parametrize("ng", [0, 1, 2, 3])
def test_massless_colour_ordered_amplitudes_parke_taylor(orc, ng):
    """Massless limit (m_t = 0) against the Parke-Taylor closed form (Phys. Rev. Lett. 56 (1986) 2459;
    with one quark line, Mangano-Parke, Phys. Rep. 200 (1991) 301, Sec. 3), all particles outgoing
    (incoming gluons: momentum and helicity reversed):
      * a quark line of equal helicities, or gluons all of one helicity: every A(sigma) vanishes;
      * exactly one gluon j of helicity -1 (or exactly one of +1): for every ordering sigma
        |A(sigma)|^2 = (2 g^2)^K s_{a j}^3 s_{b j} / (s_{t s1} s_{s1 s2} ... s_{sK tbar} s_{tbar t}),
        s_{xy} = |2 p_x.p_y|, (a, b) = (negative, positive) quark for the one negative gluon and
        (positive, negative) quark for the one positive gluon; the factor 2^K is the sqrt(2) per
        gluon of Tr(T^a T^b) = delta^ab / 2.
    A closed form for every colour-ordered amplitude of these helicities, normalisation included."""
    K, npar = ng + 2, ng + 4
    g2 = 4 * math.pi * AS
    gpart = [0, 1] + [4 + i for i in range(ng)]   # particle of gluon label 0..K-1 (order g1 g2 t tbar g3 ..)
    perms = list(permutations(range(K)))          # jamp index = lexicographic rank of the ordering
    mom, _, _ = orc.events(ng, 70 + ng, 2, mt=0.0)
    checked = 0
    for p in mom:
        mh, J = orc.me_hel(ng, p, mt=0.0, want_jamps=True)
        scale = np.abs(J).max()

        def s(a, b):
            return abs(2 * _mdot(p[a], p[b]))

        for h in range(1 << npar):
            lam = [1 if (h >> (npar - 1 - i)) & 1 else -1 for i in range(npar)]
            out = [-lam[0], -lam[1]] + lam[2:]    # all outgoing
            gl = [out[q] for q in gpart]
            nneg = gl.count(-1)
            if out[2] == out[3] or nneg in (0, K):
                assert np.abs(J[h]).max() <= 1e-10 * scale
                continue
            if nneg != 1 and nneg != K - 1:
                continue                          # beyond MHV: no one-line closed form
            odd = -1 if nneg == 1 else 1
            j = gpart[gl.index(odd)]
            qneg = 2 if out[2] < 0 else 3
            qpos = 5 - qneg
            a, b = (qneg, qpos) if odd < 0 else (qpos, qneg)
            for c, sig in enumerate(perms):
                chain = [2] + [gpart[g] for g in sig] + [3]
                den = np.prod([s(chain[i], chain[i + 1]) for i in range(len(chain) - 1)]) * s(3, 2)
                want = (2 * g2) ** K * s(a, j) ** 3 * s(b, j) / den
                assert abs(abs(J[h, c]) ** 2 / want - 1) <= 1e-10
                checked += 1
    assert checked >= 2 * math.factorial(K) * 2 * K   # at least the one-negative and one-positive sets


def _with_soft_gluon(p, lam, nhat):
    """The event p plus an outgoing gluon k = lam (sqrt(s)/2) (1, nhat), momentum conserved: the beams
    rescaled to E = k0 + sqrt(s + k0^2) and the final state boosted to total momentum (E - k0, -k)."""
    s = _mdot(p[0] + p[1], p[0] + p[1])
    k0 = lam * math.sqrt(s) / 2
    k = np.array([k0, *(k0 * nhat)])
    E = k0 + math.sqrt(s + k0 * k0)
    beta = -k[1:] / (E - k0)
    b2 = beta @ beta
    g = 1 / math.sqrt(1 - b2)
    out = np.zeros((p.shape[0] + 1, 4))
    out[0] = [E / 2, 0, 0, E / 2]
    out[1] = [E / 2, 0, 0, -E / 2]
    for i in range(2, p.shape[0]):
        bp = beta @ p[i, 1:]
        out[i, 0] = g * (p[i, 0] + bp)
        out[i, 1:] = p[i, 1:] + ((g - 1) * bp / b2) * beta + g * p[i, 0] * beta
    out[-1] = k
    return out


@pytest.mark.parametrize("ng", [0, 1, 2])
def test_soft_gluon_limit_of_colour_ordered_amplitudes(orc, ng):
    """Soft-gluon theorem for colour-ordered amplitudes (e.g. Mangano-Parke, Phys. Rep. 200 (1991)
    301, Sec. 3; Dixon, TASI'95): a gluon k inserted between colour neighbours a and b of the ordering
    (the quark line's ends included) factorises as k -> 0,
        sum over its helicities |A_{n+1}(.. a, k, b ..)|^2 -> g^2 (-J^2) |A_n(.. a, b ..)|^2,
        J = p_a / (p_a.k) - p_b / (p_b.k),
    massive tops included, for every helicity of the n other particles, every ordering and every
    insertion.  The deviation falls linearly with the soft scale: this ties each process to the one
    with a gluon less (gg->ttggg to gg->ttgg, which the brute-force Feynman-rule test pins)."""
    K, npar = ng + 2, ng + 4
    g2 = 4 * math.pi * AS
    p, _, _ = orc.events(ng, 80 + ng, 1)
    p = p[0]
    nhat = np.random.default_rng(5).normal(size=3)
    nhat /= np.linalg.norm(nhat)
    _, Jn = orc.me_hel(ng, p, want_jamps=True)
    gpart = [0, 1] + [4 + i for i in range(ng)] + [4 + ng]   # particle of gluon label; label K = the soft one
    perms_n = list(permutations(range(K)))
    rank_m = {sg: i for i, sg in enumerate(permutations(range(K + 1)))}
    big = np.abs(Jn) ** 2 >= 1e-3 * (np.abs(Jn) ** 2).max()

    def worst(lam):
        q = _with_soft_gluon(p, lam, nhat)
        assert np.abs(q[0] + q[1] - q[2:].sum(0)).max() <= 1e-9
        _, Jm = orc.me_hel(ng + 1, q, want_jamps=True)
        k = q[-1]
        dev, n = 0.0, 0
        for h in range(1 << npar):
            for c, sig in enumerate(perms_n):
                if not big[h, c]:
                    continue
                chain = [2] + [gpart[x] for x in sig] + [3]
                for pos in range(K + 1):
                    a, b = chain[pos], chain[pos + 1]
                    J = q[a] / _mdot(q[a], k) - q[b] / _mdot(q[b], k)
                    sm = list(sig)
                    sm.insert(pos, K)
                    cm = rank_m[tuple(sm)]
                    num = abs(Jm[2 * h, cm]) ** 2 + abs(Jm[2 * h + 1, cm]) ** 2   # soft gluon: last helicity bit
                    dev = max(dev, abs(num / (g2 * -_mdot(J, J) * abs(Jn[h, c]) ** 2) - 1))
                    n += 1
        return dev, n

    d4, n = worst(1e-4)
    d5, _ = worst(1e-5)
    assert n >= (1 << npar) * (K + 1)
    assert d5 <= 1e-3 and d5 <= 0.2 * d4   # the limit is reached, linearly in the soft scale


@pytest.mark.parametrize("ng", [0, 1, 2, 3])
def test_gauge_invariance(orc, ng):
    """epsilon_g -> k_g for any one gluon makes every colour-ordered amplitude vanish."""
    mom, _, _ = orc.events(ng, 50 + ng, 1)
    _, J = orc.me_hel(ng, mom[0], want_jamps=True)
    scale = np.abs(J).max()
    for g in range(ng + 2):
        _, Jg = orc.me_hel(ng, mom[0], gauge_gluon=g, want_jamps=True)
        assert np.abs(Jg).max() <= 1e-10 * scale


def _boost_rotate(p, seed):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    out = p.copy()
    out[..., 1:] = p[..., 1:] @ q.T
    beta = rng.uniform(-0.4, 0.4, size=3)
    b2 = beta @ beta
    g = 1 / math.sqrt(1 - b2)
    E, v = out[..., 0].copy(), out[..., 1:].copy()
    bp = v @ beta
    out[..., 0] = g * (E + bp)
    out[..., 1:] = v + ((g - 1) * bp / b2)[..., None] * beta + (g * E)[..., None] * beta
    return out


@pytest.mark.parametrize("ng", [0, 1, 2, 3])
def test_lorentz_invariance(orc, ng):
    mom, _, _ = orc.events(ng, 60 + ng, 2)
    for e in range(2):
        a = orc.me_hel(ng, mom[e]).sum()
        b = orc.me_hel(ng, _boost_rotate(mom[e], e)).sum()
        assert abs(b / a - 1) < 1e-12


@pytest.mark.parametrize("ng", [0, 1, 2, 3])
def test_beam_swap_and_gluon_permutation(orc, ng):
    mom, _, _ = orc.events(ng, 70 + ng, 1)
    p = mom[0]
    a = orc.me_hel(ng, p).sum()
    ps = p.copy()
    ps[[0, 1]] = ps[[1, 0]]
    ps[:, 3] *= -1
    assert abs(orc.me_hel(ng, ps).sum() / a - 1) < 1e-12
    fin = list(range(4, 4 + ng))
    for perm in list(permutations(fin))[1:3]:
        pp = p.copy()
        pp[fin] = p[list(perm)]
        assert abs(orc.me_hel(ng, pp).sum() / a - 1) < 1e-12


@pytest.mark.parametrize("ng", [1, 2])
def test_parity(orc, ng):
    """QCD conserves parity: |M_h(p)|^2 = |M_{-h}(P p)|^2 with P: p -> -p (3-momenta)."""
    mom, _, _ = orc.events(ng, 80 + ng, 1)
    p = mom[0]
    pp = p.copy()
    pp[:, 1:] *= -1
    a = orc.me_hel(ng, p)
    b = orc.me_hel(ng, pp)
    nh = len(a)
    flipped = np.array([b[(nh - 1) ^ h] for h in range(nh)])
    assert np.max(np.abs(a - flipped)) <= 1e-12 * a.max()


def test_ggtt_helicity_zeros(orc):
    """gg -> t tbar: equal physical gluon helicities (J_z = 0) produce equal-helicity top pairs only;
    the four configurations with lambda_1 = lambda_2 and lambda_t != lambda_tbar vanish."""
    mom, _, _ = orc.events(0, 5, 16)
    for e in range(16):
        mh = orc.me_hel(0, mom[e])
        zero = [h for h in range(16) if ((h >> 3) & 1) == ((h >> 2) & 1) and ((h >> 1) & 1) != (h & 1)]
        assert zero == [1, 2, 13, 14]
        for h in range(16):
            if h in zero:
                assert mh[h] <= 1e-25 * mh.sum()
            else:
                assert mh[h] > 1e-8 * mh.sum()


def test_fullcolour_wavefunctions_are_helicity_eigenstates():
    """The brute-force wavefunctions carry the physical helicities they are labelled with:
    (Sigma.p^) u = lam u, (Sigma.p^) v = -lam v, (S.k^) eps = lam eps, plus the Dirac equations."""
    from oracle import fullcolour as fc
    rng = np.random.default_rng(3)
    sig = fc._S[1:]
    for _ in range(10):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        pabs = rng.uniform(10, 700)
        p = np.concatenate([[math.sqrt(pabs**2 + MT**2)], pabs * d])
        Sig = sum(d[i] * np.kron(np.eye(2), sig[i]) for i in range(3))
        pslash = np.einsum("m,mst->st", fc.METRIC @ p, fc.GAMMA)
        for lam in (1, -1):
            u = fc.spinor_u(p, MT, lam)
            v = fc.spinor_v(p, MT, lam)
            assert np.allclose(Sig @ u, lam * u, atol=1e-9 * np.abs(u).max())
            assert np.allclose(Sig @ v, -lam * v, atol=1e-9 * np.abs(v).max())
            assert np.allclose((pslash - MT * np.eye(4)) @ u, 0, atol=1e-9 * pabs * np.abs(u).max())
            assert np.allclose((pslash + MT * np.eye(4)) @ v, 0, atol=1e-9 * pabs * np.abs(v).max())
            k = np.concatenate([[pabs], pabs * d])
            e = fc.polarisation(k, lam)
            S = [np.array([[0, 0, 0], [0, 0, -1j], [0, 1j, 0]]), np.array([[0, 0, 1j], [0, 0, 0], [-1j, 0, 0]]),
                 np.array([[0, -1j, 0], [1j, 0, 0], [0, 0, 0]])]
            Sk = sum(d[i] * S[i] for i in range(3))
            assert np.allclose(Sk @ e[1:], lam * e[1:], atol=1e-12)
            assert abs(fc.METRIC @ k @ e) < 1e-9 * pabs
            assert abs(e @ fc.METRIC @ e.conj() + 1) < 1e-12


def test_diagram_counts():
    """All tree diagrams of g g -> t tbar + n g: 3, 16, 123, 1240 (the process set of the paper)."""
    from oracle import fullcolour as fc
    golden = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "process_sizes.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                ng, nd, nh, nc = map(int, line.split())
                golden[ng] = (nd, nh, nc)
    for ng, (nd, nh, nc) in golden.items():
        assert fc.count_diagrams(ng + 2) == nd
        assert 1 << (ng + 4) == nh
        assert math.factorial(ng + 2) == nc


# ----------------------------------------------------------------------------------------
# colour matrix
# ----------------------------------------------------------------------------------------
def _numeric_colour_rows(k, rows):
    from oracle import fullcolour as fc
    perms = list(permutations(range(k)))
    # (T^sigma)_{ij} for every assignment of adjoint indices: shape [8]*k + [3,3]
    def word(sig):
        out = None
        for pos, g in enumerate(sig):
            # T^{a_g} with a_g on axis g
            shp = [1] * k + [3, 3]
            shp[g] = 8
            t = fc.T.reshape(shp)
            out = t if out is None else np.einsum("...ij,...jk->...ik", out, t)
        return np.broadcast_to(out, (8,) * k + (3, 3))
    W = {s: word(s) for s in perms}
    res = {}
    for r in rows:
        s = perms[r]
        res[r] = np.array([np.sum(W[s] * W[t].conj()).real for t in perms])
    return res


@pytest.mark.parametrize("k,rows", [(2, [0, 1]), (3, list(range(6))), (4, [0, 7, 23]), (5, [0, 77])])
def test_colour_matrix_exact_vs_gell_mann(k, rows):
    from oracle import colour
    C = colour.colour_matrix_exact(k)
    num = _numeric_colour_rows(k, rows)
    for r, vals in num.items():
        exact = np.array([float(x) for x in C[r]])
        assert np.max(np.abs(vals - exact)) < 1e-12 * np.abs(exact).max()


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_colour_matrix_structure(k):
    """Diagonal N C_F^k; symmetric; positive definite; ggtt = (1/3)[[16,-2],[-2,16]]."""
    from oracle import colour
    C = colour.colour_matrix_exact(k)
    n = len(C)
    diag = 3 * Fraction(4, 3) ** k
    for i in range(n):
        assert C[i][i] == diag
        for j in range(i):
            assert C[i][j] == C[j][i]
    ev = np.linalg.eigvalsh(colour.colour_matrix(k))
    assert ev.min() > 0
    if k == 2:
        assert C == ((Fraction(16, 3), Fraction(-2, 3)), (Fraction(-2, 3), Fraction(16, 3)))


# ----------------------------------------------------------------------------------------
# helicity filter and flop counter
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("ng,nwarm", [(0, 1024), (1, 1024), (2, 256), (3, 64)])
def test_helicity_filter_gap(orc, ng, nwarm):
    """Rejected and accepted max-ratios are at least six decades apart around tau = 1e-9, so the
    mask cannot depend on FP rounding order."""
    mom, _, _ = orc.events(ng, 1 + ng, nwarm)
    mask, ratio = orc.hel_mask(ng, mom, nthreads=os.cpu_count() or 1)
    acc = ratio[ratio > 1e-9]
    rej = ratio[ratio <= 1e-9]
    # accepted ratios sit >= 2 decades above tau, rejected ones (exact zeros up to rounding)
    # >= 6 decades below it
    assert acc.min() > 1e-7
    if len(rej):
        assert rej.max() < 1e-15
        assert acc.min() / rej.max() > 1e6
    expect_good = 12 if ng == 0 else 1 << (ng + 4)
    assert len(acc) == expect_good
    bits = sum(bin(int(w)).count("1") for w in mask)
    assert bits == expect_good


@pytest.mark.parametrize("ng", [0, 1, 2])
def test_flop_counter_colour_part(orc, ng):
    """The colour sum costs exactly 4 ncol^2 + 4 ncol flops per helicity."""
    mom, _, _ = orc.events(ng, 1, 1)
    c = orc.flops(ng, mom[0])
    ncol = math.factorial(ng + 2)
    nh = 1 << (ng + 4)
    assert c["colour"]["add"] + c["colour"]["mul"] == nh * (4 * ncol * ncol + 4 * ncol)
    assert c["amp"]["add"] + c["amp"]["mul"] > 0


# ------------------------------------------------------------------------------------------
# The oracle's amplitude operation counter, pinned to a count derived by hand from the algorithm:
# per helicity, the external wavefunctions, every off-shell gluon current J(seq) once per ordered
# sequence of distinct gluons (length L = 2..k: k!/(k-L)! of them), every quark-line prefix
# Psibar(prefix) once per ordered prefix (length 1..k-1), and k terms per colour ordering (k! of them).
# Costs per primitive, with a complex add = 2 adds and a complex multiply = 4 mul + 2 add:
#   dot_cc 16 mul 14 add; dot_cr 8 mul 6 add; dot_rr 4 mul 3 add;
#   row spinor x (gamma.J): the two J1 -+ i J2 (8 mul 4 add), eight complex sums or differences
#   (16 add), four outputs of two complex products and a sum (32 mul 24 add) -> 40 mul 44 add;
#   row spinor x (Qslash + m): 40 mul 44 add + 4 (scale, complex add) -> 48 mul 52 add.
# ------------------------------------------------------------------------------------------
def _hand_amp_count(k, mt_nonzero=True):
    """(add, mul) per helicity of the oracle's colour-ordered recursion for k gluons (massive tops,
    incoming gluons along the beam, final-state gluons off the axis)."""
    from math import comb, factorial
    nseq = lambda L: factorial(k) // factorial(k - L)
    add = mul = 0
    # ubar(p_t) and v(p_tbar): |p| (3 mul 2 add), E + |p| (1 add), m*m (1 mul), the helicity
    # spinor chi (3 mul 2 add for pt^2 and |p|, one add for |p| + pz, 2 mul for 2|p|(|p| + pz),
    # 3 mul for its components), four scaled components (8 mul)
    add += 2 * (2 + 1 + 3)
    mul += 2 * (3 + 1 + 8 + 8)
    # gluon polarisations: kt (2 mul 1 add), |k| (3 mul 2 add), 1/sqrt(2) scalings (6 mul); off the
    # beam axis also e_theta, e_phi (4 mul)
    for g in range(k):
        add += 3
        mul += 2 + 3 + 6 + (4 if g >= 2 else 0)
    mul += 1                                                      # g_s = sqrt(4 pi alpha_s)
    for L in range(2, k + 1):                                     # off-shell gluon currents
        n3, n4 = L - 1, comb(L - 1, 2)
        # momentum sum 4L add; three-gluon split: dot_cc, d / a1 / a2 (8 mul 12 add), two dot_cr,
        # four components of (scale + 2 complex products, 3 complex sums, g scaling) = 88 mul 78 add;
        # four-gluon split: three dot_cc, four components of (3 complex products, 2 scalings, 2 sums,
        # g*g, g^2 scaling, accumulation) = 116 mul 90 add; propagator dot_rr + 4 scalings
        add += nseq(L) * (4 * L + 78 * n3 + 90 * n4 + 3)
        mul += nseq(L) * (88 * n3 + 116 * n4 + 4 + 8)
    for ln in range(1, k):                                        # quark-line prefixes
        # per attached current: row x gamma.J + i g scaling and accumulation (48 mul 52 add); momentum
        # Q (4 len add); (Qslash + m) (48 mul 52 add); Q^2 - m^2 (5 mul 4 add), m w (1 mul), the
        # propagator's 1/|d|^2 (2 mul 1 add) and its two components (2 mul); times the spinor (16 mul 8 add)
        add += nseq(ln) * (52 * ln + 4 * ln + 52 + 4 + 1 + 8)
        mul += nseq(ln) * (48 * ln + 48 + 5 + 1 + 2 + 2 + 16)
    # amplitude terms: row x gamma.J, the product with v (16 mul 14 add), i g scaling and sum (2 mul 2 add)
    add += factorial(k) * k * (44 + 14 + 2)
    mul += factorial(k) * k * (40 + 16 + 2)
    return add, mul


@pytest.mark.parametrize("ng", [0, 1, 2, 3])
def test_flop_counter_amplitude_part_hand_count(orc, ng):
    """The oracle's amplitude counts equal the count derived by hand from the algorithm (every add and
    multiply of the recursion, exact), for one helicity and for every helicity of a mask: the count
    scales with the number of good helicities and nothing else."""
    mom, _, _ = orc.events(ng, 7, 1)
    add1, mul1 = _hand_amp_count(ng + 2)
    nhel = 1 << (ng + 4)
    one = np.zeros((nhel + 31) // 32, dtype=np.uint32)
    one[0] = 1
    c1 = orc.flops(ng, mom[0], mask=one)
    assert (c1["amp"]["add"], c1["amp"]["mul"]) == (add1, mul1)
    rng = np.random.default_rng(ng)
    hs = rng.choice(nhel, size=nhel // 3 + 1, replace=False)
    m = np.zeros_like(one)
    for h in hs:
        m[h >> 5] |= np.uint32(1 << (int(h) & 31))
    c = orc.flops(ng, mom[0], mask=m)
    assert (c["amp"]["add"], c["amp"]["mul"]) == (len(hs) * add1, len(hs) * mul1)
    ncol = math.factorial(ng + 2)
    assert c["colour"]["add"] == c["colour"]["mul"] == len(hs) * (2 * ncol * ncol + 2 * ncol)


def test_oracle_flops_golden_is_the_oracles_count(orc):
    """tests/golden/oracle_flops.txt (the roofline numerator bench.py reads) is what the oracle counts
    now, and each amplitude count is good helicities x the hand-derived per-helicity count."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(os.path.dirname(__file__), "golden",
                                                                     "make_oracle_flops.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    stored = [ln.split() for ln in open(mk.OUT) if ln.strip() and not ln.startswith("#")]
    fresh = [[str(x) for x in r] for r in mk.rows()]
    assert stored == fresh
    for r in fresh:
        ng, good, add, mul = int(r[1]), int(r[2]), int(r[3]), int(r[4])
        a1, m1 = _hand_amp_count(ng + 2)
        assert (add, mul) == (good * a1, good * m1)
