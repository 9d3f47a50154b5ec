"""GPU parity with a partial helicity mask: the CUDA path through the C ABI against the FP64 CPU oracle
when a helicity threshold keeps only part of the helicities (arXiv 2210.11122 Sec. 2: the helicity
filter only skips helicities; every kept one is summed exactly as in the full sum).

Kept in a file of its own that runs after the other GPU tests.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SQRTS = 1500.0
NTHREADS = os.cpu_count() or 1
# n_g -> (seed, events for element-by-element parity, full workload size), as the parity tests
WORKLOADS = {0: (1, 16384, 16384), 1: (2, 4099, 524288), 2: (3, 1027, 262144), 3: (4, 131, 65536)}


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


@pytest.mark.parametrize("ng", [1, 2, 3])
def test_partial_helicity_mask_every_mode(env, ng):
    """A helicity threshold between the oracle's per-helicity maximum ratios keeps about half of the
    helicities: fewer gluon-helicity slots than combinations, slots with only some good top helicities,
    and tensor-core rows past the last good slot.  The GPU gets the oracle's own momenta, so both sides
    see identical inputs.  The mask equals the oracle's at that threshold; plain FP64 matches the oracle
    with that mask within 1e-12 per event, relative to the partial (masked) sum itself, which is a sum of
    positive per-helicity terms; the other modes (and kernel variants) stay within their bounds of FP64,
    relative to the event's full matrix element."""
    torch, mg, orc = env
    seed = WORKLOADS[ng][0]
    n = 131 if ng == 3 else 257   # the filter's warm-up is the whole (ragged) batch
    evs, _, _ = orc.events(ng, seed, n)
    _, ratio = orc.hel_mask(ng, evs, nthreads=NTHREADS)
    r = np.sort(ratio[ratio > 0])
    mid = len(r) // 2
    k = max(range(mid - len(r) // 4, mid + len(r) // 4), key=lambda i: r[i + 1] / r[i])   # widest gap
    tau = float(np.sqrt(r[k] * r[k + 1]))
    ref_mask, _ = orc.hel_mask(ng, evs, tau=tau, nthreads=NTHREADS)
    nhel = 1 << (ng + 4)
    ngood_ref = sum(bin(int(w)).count("1") for w in ref_mask)
    assert 0 < ngood_ref < nhel
    ref = orc.me_batch(ng, evs, mask=ref_mask, nthreads=NTHREADS)
    full = orc.me_batch(ng, evs, nthreads=NTHREADS)
    with mg.Context(ng, hel_warmup=n, hel_tau=tau) as ctx:
        mom = torch.from_numpy(mg.to_aosoa(evs)).cuda()
        me = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        ctx.hel_filter(mom, n)
        ctx.sigmakin(mom, n, me, mg.MG_FP64)
        gmask, ngood = ctx.hel_mask()
        assert np.array_equal(gmask, ref_mask) and ngood == ngood_ref
        fp64 = me.cpu().numpy()
        assert np.all(fp64 > 0)
        rel = np.abs(fp64 / ref - 1)
        assert rel.max() <= 1e-12, (rel.max(), int(np.argmax(rel)))
        for flags in (39, 7):   # FP64 with and without the currents shared between slots
            ctx.set_launch_shape(mg.MG_FP64, 128, 0, flags)
            ctx.sigmakin(mom, n, me, mg.MG_FP64)
            rel = np.abs(me.cpu().numpy() / ref - 1)
            assert rel.max() <= 1e-12, (flags, rel.max(), int(np.argmax(rel)))
        variants = [(mg.MG_FP64_TCCOLOR, None, 1e-6), (mg.MG_FP32_AMP, None, 1e-5), (mg.MG_MIXED, None, 1e-5)]
        if ng >= 2:   # lane-group kernel: in-kernel and separate tensor-core colour sums
            variants += [(mg.MG_MIXED, 15, 1e-5), (mg.MG_MIXED, 31, 1e-5)]
        for prec, flags, bound in variants:
            if flags is not None:
                ctx.set_launch_shape(prec, 128, 0, flags)
            ctx.sigmakin(mom, n, me, prec)
            got = me.cpu().numpy()
            assert np.max(np.abs(got - fp64) / full) <= bound, (prec, flags)
