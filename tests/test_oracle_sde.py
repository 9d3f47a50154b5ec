"""CPU pins of the oracle's single-diagram-enhancement channels (oracle/sde.py; arXiv 2210.11122 Sec. 2):
the diagram counts, and the colour-ordered amplitudes of the independent Berends-Giele oracle recovered as
fixed linear combinations of the single-diagram amplitudes (every event and helicity at once), which ties
every diagram amplitude, its propagators and vertices, to the pinned matrix elements."""
import os

import numpy as np
import pytest

from oracle import sde

HERE = os.path.dirname(os.path.abspath(__file__))


def golden_counts():
    out = {}
    for line in open(os.path.join(HERE, "golden", "process_sizes.txt")):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            out[int(f[0])] = int(f[1])
    return out


@pytest.mark.parametrize("ng", [0, 1, 2, 3])
def test_channel_counts(ng):
    """Three-point-vertex diagrams 3 / 15 / 105 / 945; with the four-gluon-vertex ones added, the process's
    diagram count (3 / 16 / 123 / 1240); keys unique."""
    ch = sde.diagrams(ng)
    assert len(ch) == [3, 15, 105, 945][ng]
    assert len({sde.key(d) for d in ch}) == len(ch)
    assert len(sde.diagrams(ng, four=True)) == golden_counts()[ng]


def _fit_residual(target, basis):
    """Relative residual of the least-squares fit target ~ basis @ x (complex)."""
    x, *_ = np.linalg.lstsq(basis, target, rcond=None)
    return np.linalg.norm(basis @ x - target) / np.linalg.norm(target), x


@pytest.mark.parametrize("ng", [0, 1])
def test_colour_ordered_amplitudes_are_fixed_sums_of_diagrams(orc, ng):
    """For every colour ordering sigma, the oracle's colour-ordered amplitude A(sigma) over many events and
    helicities equals sum_d x_d A_d with constants x_d (plus, with three gluons, the three Lorentz
    structures of the four-gluon vertex on the line, (J_a.J_b) ubar gammaJ_c v / P^2): the residual is at
    rounding level, and every three-point diagram takes part in some ordering."""
    dias = sde.diagrams(ng)
    nhel = 1 << (ng + 4)
    mom, _, _ = orc.events(ng, 31, 6)
    rows, targets = [], []
    for p in mom:
        _, jamps = orc.me_hel(ng, p, want_jamps=True)
        for h in range(nhel):
            a = sde.amplitudes(ng, p, h, dias=dias)
            if np.abs(jamps[h]).max() == 0:
                continue
            extra = []
            if ng == 1:
                q, eps, ub, v = sde.externals(ng, p, h, 173.0)
                P = q[0] + q[1] + q[2]
                for (i, j, k) in ((0, 1, 2), (1, 2, 0), (0, 2, 1)):
                    J = sde._dot(eps[i], eps[j]) * eps[k] / sde._dot(P, P)
                    extra.append(ub @ sde._slash(J) @ v)
            rows.append(np.concatenate([a, extra]))
            targets.append(jamps[h])
    B = np.array(rows)
    T = np.array(targets)
    used = np.zeros(len(dias), dtype=bool)
    mods = []
    for s in range(T.shape[1]):
        res, x = _fit_residual(T[:, s], B)
        assert res < 1e-9, (s, res)
        xd = np.abs(x[: len(dias)])
        on = xd > 1e-6 * xd.max()
        used |= on
        mods.extend(xd[on])
    assert used.all()
    # the colour decomposition gives every planar diagram the coefficient (+-1 or +-i) g^(n_g+2): one
    # modulus for all, which fixes each diagram's normalisation (a wrong constant factor in one diagram,
    # invisible to the fit, would show here)
    mods = np.array(mods)
    assert np.max(np.abs(mods / mods[0] - 1)) < 1e-8, mods


def test_weights_normalised(orc):
    mom, _, _ = orc.events(1, 5, 2)
    mask, _ = orc.hel_mask(1, mom)
    for p in mom:
        w = sde.weights(1, p, mask)
        assert np.all(w > 0) and abs(w.sum() - 1) < 1e-14
