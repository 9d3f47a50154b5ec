"""One persistent launch for the FP64 matrix elements of a batch of jobs of different processes and sizes
(mg_sigmakin_batch, and graphs created with MG_GRAPH_PERSISTENT), through the C ABI: every job against the
FP64 oracle on the oracle's own momenta (1e-12 per event), and bit for bit against the one-job-per-launch
path it reorganises (mg_sigmakin with the unshared-current launch shape).  The paper's Sec. 4 motivates
it: small batches leave the GPU underfilled."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SQRTS = 1500.0
NTHREADS = os.cpu_count() or 1
UNSHARED = 7   # MG_LAUNCH_UNROLLED | DF_REDO | FUSED, no MG_LAUNCH_SHARED


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_2210_11122_gb300 as mg
    from paper_2210_11122_gb300 import build
    build.build()
    oracle.build()
    return torch, mg, oracle


# (n_g, events, seed): every process, ragged sizes, several jobs of one process
MIX = [(3, 13, 71), (0, 1000, 72), (1, 257, 73), (2, 37, 74), (1, 5, 75), (0, 33, 76), (2, 129, 77), (3, 1, 78)]


def test_batch_matches_oracle_and_single_launches(env):
    torch, mg, orc = env
    ctxs, moms, mes, refs = [], [], [], []
    try:
        for ng, n, seed in MIX:
            evs, _, _ = orc.events(ng, seed, n)
            mask, _ = orc.hel_mask(ng, evs[:1024], nthreads=NTHREADS)
            refs.append(orc.me_batch(ng, evs, mask=mask, nthreads=NTHREADS))
            c = mg.Context(ng, hel_warmup=1024)
            c.set_launch_shape(mg.MG_FP64, 128, 0, UNSHARED)
            ctxs.append(c)
            moms.append(torch.from_numpy(mg.to_aosoa(evs)).cuda())
            mes.append(torch.full((n,), -1.0, dtype=torch.float64, device="cuda"))
        mg.sigmakin_batch([(c, m, n, me) for c, m, (_, n, _), me in zip(ctxs, moms, MIX, mes)])
        for c in ctxs:
            assert c.check() == 0
        got = [me.cpu().numpy() for me in mes]
        for (ng, n, _), c, m, g, r in zip(MIX, ctxs, moms, got, refs):
            rel = np.abs(g / r - 1)
            assert rel.max() <= 1e-12, (ng, n, rel.max())
            one = torch.zeros(n, dtype=torch.float64, device="cuda")
            c.sigmakin(m, n, one, mg.MG_FP64)
            assert np.array_equal(one.cpu().numpy(), g), (ng, n)
    finally:
        for c in ctxs:
            c.close()


def test_persistent_graph_equals_branch_graph_and_updates(env):
    torch, mg, orc = env
    sizes = [(0, 3000), (1, 700), (2, 150), (3, 40), (1, 64)]
    made = []
    try:
        def jobs(seed0, persistent):
            out = []
            for i, (ng, n) in enumerate(sizes):
                c = mg.Context(ng)
                c.set_launch_shape(mg.MG_FP64, 128, 0, UNSHARED)
                made.append(c)
                mom = torch.zeros(c.mom_count(n), dtype=torch.float64, device="cuda")
                me = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
                out.append((c, seed0 + i, 0, n, SQRTS, mom, me, mg.MG_FP64))
            return out
        ja, jb = jobs(100, True), jobs(100, False)
        ga, gb = mg.GraphBatch(ja, persistent=True), mg.GraphBatch(jb)
        ga.launch()
        gb.launch()
        torch.cuda.synchronize()
        for a, b in zip(ja, jb):
            assert np.array_equal(a[6].cpu().numpy(), b[6].cpu().numpy())
        # new seeds, same topology: in-place update of both graphs
        ja2 = [(c, s + 50, e0, n, q, mom, me, p) for c, s, e0, n, q, mom, me, p in ja]
        jb2 = [(c, s + 50, e0, n, q, mom, me, p) for c, s, e0, n, q, mom, me, p in jb]
        ga.update(ja2)
        gb.update(jb2)
        ga.launch()
        gb.launch()
        torch.cuda.synchronize()
        for a, b in zip(ja2, jb2):
            assert np.array_equal(a[6].cpu().numpy(), b[6].cpu().numpy())
            assert np.all(a[6].cpu().numpy() > 0)
        ga.close()
        gb.close()
        with pytest.raises(mg.MGError):   # persistent graphs take FP64 jobs only
            mg.GraphBatch([(ja[0][0], 1, 0, 100, SQRTS, ja[0][5], ja[0][6], mg.MG_MIXED)], persistent=True)
    finally:
        for c in made:
            c.close()
