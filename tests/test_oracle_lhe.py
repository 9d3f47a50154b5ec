"""CPU pins of the oracle's event-level epilogues (oracle/lhe.py): the running coupling, the scale, the
coupling power of the tree amplitudes, and the inverse-transform choices (arXiv 2210.11122 Sec. 2:
running alpha_s; Sec. 4: event-by-event helicities and leading colours of LHE files)."""
import math

import numpy as np
import pytest

from oracle import lhe


def test_alphas_one_loop_solves_its_equation():
    """alpha_s(M_Z) is the input; the function solves d alpha / d ln mu^2 = -b0 alpha^2 with
    b0 = 23/(12 pi) for five flavours (central differences in ln mu^2), and decreases with mu."""
    assert lhe.alphas_1loop(0.118, lhe.MZ) == 0.118
    assert abs(lhe.b0() - 23.0 / (12.0 * math.pi)) < 1e-16
    d = 1e-4
    prev = None
    for mu in (20.0, 91.1876, 173.0, 500.0, 1500.0, 7000.0):
        a = lhe.alphas_1loop(0.118, mu)
        up = lhe.alphas_1loop(0.118, mu * math.exp(d / 2))
        dn = lhe.alphas_1loop(0.118, mu * math.exp(-d / 2))
        deriv = (up - dn) / (2 * d)   # ln mu^2 moves by 2 d
        assert abs(deriv / (-lhe.b0() * a * a) - 1) < 1e-7
        if prev is not None:
            assert a < prev
        prev = a
    # the closed form composes: running M_Z -> mu1 -> mu2 equals M_Z -> mu2
    a1 = lhe.alphas_1loop(0.118, 300.0)
    a2 = a1 / (1 + a1 * lhe.b0() * math.log(900.0 ** 2 / 300.0 ** 2))
    assert abs(a2 / lhe.alphas_1loop(0.118, 900.0) - 1) < 1e-14


def test_half_ht_by_hand():
    mt = 173.0
    p = np.zeros((5, 4))
    p[2, 1:3] = [30.0, 40.0]          # top: pT 50
    p[3, 1:3] = [-30.0, -40.0]        # antitop
    p[4, 1:3] = [0.0, 0.0]            # a gluon along the beam adds nothing
    assert abs(lhe.half_ht(p, mt) - math.sqrt(mt * mt + 2500.0)) < 1e-12
    p[4, 1:3] = [6.0, 8.0]            # massless gluon: its pT
    assert abs(lhe.half_ht(p, mt) - (math.sqrt(mt * mt + 2500.0) + 5.0)) < 1e-12


@pytest.mark.parametrize("ng", [0, 1, 2])
def test_tree_matrix_element_carries_alphas_to_the_power_of_the_gluon_count(orc, ng):
    """Every tree diagram of g g -> t tbar + n g has n + 2 gluon vertices' worth of g_s^2 in |M|^2: the
    oracle's full evaluation at two couplings differs by (a2/a1)^(n+2)."""
    mom, _, _ = orc.events(ng, 3, 4)
    m1 = orc.me_batch(ng, mom, alphas=0.118)
    m2 = orc.me_batch(ng, mom, alphas=0.0923)
    assert np.max(np.abs(m2 / m1 / (0.0923 / 0.118) ** (ng + 2) - 1)) < 1e-13


def test_inverse_transform_frequencies_and_ends():
    w = [0.0, 3.0, 0.5, 0.0, 1.5, 5.0]
    tot = sum(w)
    n = 10000
    counts = np.zeros(len(w), dtype=int)
    for j in range(n):
        counts[lhe.inverse_transform(w, (j + 0.5) / n)] += 1
    for i, wi in enumerate(w):
        assert abs(counts[i] - n * wi / tot) <= 1
    assert lhe.inverse_transform(w, 0.0) == 1          # first entry of nonzero weight
    assert lhe.inverse_transform(w, 1.0 - 1e-15) == 5
    assert lhe.inverse_transform([2.0], 0.7) == 0


@pytest.mark.parametrize("ng", [0, 1, 2])
def test_event_choices_follow_the_weights(orc, ng):
    """For one event, the helicity choice over stratified uniforms reproduces |M_h|^2 / sum |M_h'|^2 and
    never picks a helicity outside the mask; the colour choice reproduces w_sigma / sum w; me equals
    me_batch at the same coupling."""
    mom, _, _ = orc.events(ng, 5, 1)
    mask, _ = orc.hel_mask(ng, mom)
    me, _, _, a, det = lhe.event(ng, mom[0], mask)
    assert abs(me / orc.me_batch(ng, mom, mask=mask)[0] - 1) < 1e-14
    good, mh, w = det["good"], det["mh"], det["w"]
    n = 2000
    hc = {}
    cc = np.zeros(len(w), dtype=int)
    for j in range(n):
        r = (j + 0.5) / n
        _, h, c, _, _ = lhe.event(ng, mom[0], mask, r_hel=r, r_col=r)
        hc[h] = hc.get(h, 0) + 1
        cc[c] += 1
    tot = sum(mh[h] for h in good)
    assert set(hc) <= set(good)
    for h in good:
        assert abs(hc.get(h, 0) - n * mh[h] / tot) <= 1
    for c in range(len(w)):
        assert abs(cc[c] - n * w[c] / w.sum()) <= 1


def test_running_event_uses_the_scale(orc):
    mom, _, _ = orc.events(1, 9, 1)
    mask, _ = orc.hel_mask(1, mom)
    me_fix, _, _, a_fix, _ = lhe.event(1, mom[0], mask)
    me_run, _, _, a_run, _ = lhe.event(1, mom[0], mask, running=True)
    assert a_fix == 0.118
    assert a_run == lhe.alphas_1loop(0.118, lhe.half_ht(mom[0], 173.0))
    assert abs(me_run / me_fix / (a_run / 0.118) ** 3 - 1) < 1e-13
