"""GPU parity of the single-diagram-enhancement channel weights (mg_sde_weights; arXiv 2210.11122 Sec. 2)
against the oracle's diagram-by-diagram evaluation (oracle/sde.py, 4x4 gamma matrices, its own
wavefunctions), on the oracle's own momenta and helicity mask; channels matched by key."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import oracle.sde as osde
    import paper_2210_11122_gb300 as mg
    from paper_2210_11122_gb300 import build
    build.build()
    oracle.build()
    return torch, mg, oracle, osde


@pytest.mark.parametrize("ng,nevt,ncheck", [(0, 97, 97), (1, 41, 41), (2, 19, 6), (3, 35, 2)])
def test_sde_weights_match_oracle(env, ng, nevt, ncheck):
    torch, mg, orc, osde = env
    evs, _, _ = orc.events(ng, 90 + ng, nevt)
    mask, _ = orc.hel_mask(ng, evs, nthreads=NTHREADS)
    keys = mg.sde_channels(ng)
    nch = len(keys)
    with mg.Context(ng, hel_warmup=nevt) as ctx:
        mom = torch.from_numpy(mg.to_aosoa(evs)).cuda()
        ctx.hel_filter(mom, nevt)
        w = torch.full((nch * nevt,), -1.0, dtype=torch.float64, device="cuda")
        ctx.sde_weights(mom, nevt, w)
        assert ctx.check() == 0
        got = w.cpu().numpy().reshape(nch, nevt)
    assert np.all(got >= 0) and np.max(np.abs(got.sum(axis=0) - 1)) < 1e-13
    dias = osde.diagrams(ng)
    pos = {osde.key(d): i for i, d in enumerate(dias)}
    order = [pos[k] for k in keys]
    for e in np.linspace(0, nevt - 1, ncheck).astype(int):
        ref = osde.weights(ng, evs[e], mask, dias=dias)[order]
        assert np.max(np.abs(got[:, e] - ref)) <= 1e-12 * ref.max(), (e, np.max(np.abs(got[:, e] - ref)))
        big = ref > 1e-6 * ref.max()
        assert np.max(np.abs(got[big, e] / ref[big] - 1)) <= 1e-10
