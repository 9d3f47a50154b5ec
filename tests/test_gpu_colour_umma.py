"""The separate tensor-core colour pass on the fifth-generation tensor cores (tcgen05.mma, accumulators in
tensor memory; the default) against the FP64 oracle and against the warp-level mma.sync pass
(MG_LAUNCH_TC_SYNC), through the C ABI.  The colour decomposition (Mangano-Parke) makes the colour sum
of a helicity the quadratic form A^dagger C A with the exact colour matrix C; the tensor cores compute it
with C exact in FP16 and each jamp row split into two FP16 values (~2^-24 of the row maximum), FP32
accumulation: per-helicity relative error ~1e-7, so 1e-6 per event is the bar for FP64 amplitudes and
1e-5 for FP32 amplitudes (the amplitudes' own error).
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SQRTS = 1500.0
NTHREADS = os.cpu_count() or 1


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


@pytest.mark.parametrize("ng,nevt", [(0, 1031), (1, 517), (2, 131), (3, 29)])
def test_umma_colour_pass_matches_oracle_and_mma_sync(env, ng, nevt):
    torch, mg, orc = env
    evs, _, _ = orc.events(ng, 60 + ng, nevt)
    mask, _ = orc.hel_mask(ng, evs[:1024], nthreads=NTHREADS)
    ref = orc.me_batch(ng, evs, mask=mask, nthreads=NTHREADS)
    got = {}
    with mg.Context(ng) as ctx:
        mom = torch.from_numpy(mg.to_aosoa(evs)).cuda()
        me = torch.full((nevt,), -1.0, dtype=torch.float64, device="cuda")
        for prec, base in ((mg.MG_FP64_TCCOLOR, 7), (mg.MG_MIXED, 7 | mg.LAUNCH_TC_APART | mg.LAUNCH_WARP)):
            for sync in (0, mg.LAUNCH_TC_SYNC):
                ctx.set_launch_shape(prec, 128, 0, base | sync)
                ctx.sigmakin(mom, nevt, me, prec)
                assert ctx.check() == 0
                got[(prec, sync)] = me.cpu().numpy().copy()
    for (prec, sync), g in got.items():
        bound = 1e-6 if prec == mg.MG_FP64_TCCOLOR else 1e-5
        rel = np.abs(g / ref - 1)
        assert np.all(np.isfinite(g)) and rel.max() <= bound, (prec, sync, rel.max())
    for prec in (mg.MG_FP64_TCCOLOR, mg.MG_MIXED):
        a, b = got[(prec, 0)], got[(prec, mg.LAUNCH_TC_SYNC)]
        assert np.max(np.abs(a / b - 1)) <= 2e-6


def test_umma_colour_pass_full_size(env):
    """gg->ttggg at its workload size (65,536 events, every helicity): the FP64-amplitude tensor-core mode
    against plain FP64 on the same momenta, every event."""
    torch, mg, orc = env
    n = 65536
    with mg.Context(3) as ctx:
        mom = torch.zeros(ctx.mom_count(n), dtype=torch.float64, device="cuda")
        ctx.rambo(4, n, SQRTS, mom)
        a = torch.zeros(n, dtype=torch.float64, device="cuda")
        b = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.sigmakin(mom, n, a, mg.MG_FP64)
        ctx.sigmakin(mom, n, b, mg.MG_FP64_TCCOLOR)
        assert ctx.check() == 0
        rel = (b / a - 1).abs().max().item()
    assert rel <= 1e-6, rel


def test_umma_bounded_wait_reports_timeout_and_context_recovers(env):
    """The failure path of the tensor-memory colour pass without a fault: with MMAs withheld
    (mg_diag_tc_stall) every CTA's bounded mbarrier wait runs out after 0.2 s; the kernel records it,
    frees its tensor memory and returns; mg_check reports MG_ETIMEOUT once; then, back to normal, the
    same context gives the same values as before."""
    torch, mg, orc = env
    n = 4096
    with mg.Context("ggttgg") as ctx:
        mom = torch.zeros(ctx.mom_count(n), dtype=torch.float64, device="cuda")
        ctx.rambo(9, n, SQRTS, mom)
        ctx.set_launch_shape(mg.MG_FP64_TCCOLOR, 128, 0, 7)
        a = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.sigmakin(mom, n, a, mg.MG_FP64_TCCOLOR)
        assert ctx.check() == 0
        ctx.diag_tc_stall(True)
        b = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.sigmakin(mom, n, b, mg.MG_FP64_TCCOLOR)
        with pytest.raises(mg.MGError) as e:
            ctx.check()
        assert e.value.status == 6
        assert ctx.check() == 0                     # the flag was read and cleared
        ctx.diag_tc_stall(False)
        c = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.sigmakin(mom, n, c, mg.MG_FP64_TCCOLOR)
        assert ctx.check() == 0
        assert torch.equal(a, c)


def test_mma_peak_microbenchmark_is_exact_and_plausible(env):
    """The tensor-core microbenchmark (tcgen05.mma kind::f16, the colour pass's instruction): the library
    checks the accumulated integer products exactly; the rate lies between a tenth of and 1.5x the
    nominal dense FP16 peak of 2.25 PFLOP/s."""
    torch, mg, orc = env
    r = mg.measure_mma_peak(4096)
    assert 2.25e14 < r < 3.4e15, r
