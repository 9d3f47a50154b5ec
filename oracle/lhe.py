"""Event-level epilogues of the FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Plain definitions, one event at a time, on top of me_oracle.cpp's per-helicity colour sums and
colour-ordered amplitudes (jamps):

  * running coupling (arXiv 2210.11122 Sec. 2 lists the "running" of alpha_s among the engine's features):
    one-loop solution of d alpha / d ln mu^2 = -b0 alpha^2, b0 = (33 - 2 n_f) / (12 pi), from
    alpha_s(M_Z); the scale is mu = H_T / 2, half the sum of the final-state transverse masses.  The
    oracle evaluates the whole matrix element with g_s = sqrt(4 pi alpha_s(mu)) (it does not use the
    coupling power law that the GPU epilogue relies on, so the two are independent);
  * helicity choice for an unweighted event (Sec. 4: event-by-event helicities missing from the LHE
    files): helicity h with probability |M_h|^2 / sum_h' |M_h'|^2 over the good helicities, by inverse
    transform of a caller's uniform r: the smallest good h (ascending index) whose running sum exceeds
    r times the total;
  * leading-colour choice (Sec. 4: leading colours missing from the LHE files): colour flow sigma with
    probability w_sigma / sum w, w_sigma = sum over good helicities of |J_sigma(h)|^2, by the same inverse
    transform over sigma in lexicographic order.
"""
import math

import numpy as np

from . import me_hel, nhel

MZ = 91.1876
NF = 5


def b0(nf=NF):
    return (33.0 - 2.0 * nf) / (12.0 * math.pi)


def alphas_1loop(alphas_mz, mu, nf=NF, mz=MZ):
    """One-loop running coupling at scale mu from alpha_s(M_Z)."""
    return alphas_mz / (1.0 + alphas_mz * b0(nf) * math.log(mu * mu / (mz * mz)))


def half_ht(p, mt):
    """H_T / 2 of one event p[npar][4] (particle order g1 g2 t tbar g3..): half the sum over the
    final-state particles of sqrt(m^2 + px^2 + py^2)."""
    ht = 0.0
    for i in range(2, len(p)):
        m = mt if i < 4 else 0.0
        ht += math.sqrt(m * m + p[i][1] ** 2 + p[i][2] ** 2)
    return 0.5 * ht


def inverse_transform(weights, r):
    """Index of the first weight whose running sum exceeds r times the total (the last one if rounding
    leaves none); weights are visited in the order given."""
    total = 0.0
    for w in weights:
        total += w
    target = r * total
    cum = 0.0
    for i, w in enumerate(weights):
        cum += w
        if cum > target:
            return i
    return len(weights) - 1


def event(ng, p, mask, r_hel=None, r_col=None, running=False, mt=173.0, alphas=0.118):
    """One event: (me, chosen helicity or None, chosen colour flow or None, alpha_s used, details).
    me is averaged as me_batch: (1/256)(1/ng!) sum over the good helicities of the colour sums."""
    a = alphas_1loop(alphas, half_ht(p, mt)) if running else alphas
    mh, jamps = me_hel(ng, p, mt=mt, alphas=a, want_jamps=True)
    good = [h for h in range(nhel(ng)) if (int(mask[h >> 5]) >> (h & 31)) & 1]
    me = sum(mh[h] for h in good) / (256.0 * math.factorial(ng))
    hel = good[inverse_transform([mh[h] for h in good], r_hel)] if r_hel is not None else None
    w = np.zeros(jamps.shape[1])
    for h in good:
        w += jamps[h].real ** 2 + jamps[h].imag ** 2
    col = inverse_transform(list(w), r_col) if r_col is not None else None
    return me, hel, col, a, {"mh": mh, "good": good, "w": w}
