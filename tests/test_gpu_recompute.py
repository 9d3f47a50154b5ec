"""The FP32 modes' recomputation of events with a small internal invariant, forced onto every event
(recomputation threshold tau = 1: every internal invariant is below s), through the C ABI.

With four and five gluons the recomputation is the lane-group kernel with double-float amplitudes
(~48 bits) and an FP32 colour sum on the jamps rounded to FP32; with fewer gluons the per-thread
double-float kernel.  Its error is then that of the FP32 colour sum alone: the colour matrix is exact
and the quadratic form well conditioned (condition number <= 16), so each jamp's FP32 rounding
(2^-24) moves a colour sum by at most ~2e-6 relative, far below the plain-FP32 amplitudes' error.
Compared per event with plain FP64 on the oracle's own momenta, and with the oracle on a sample, in
both output layouts: per slot (FP32 amplitudes) and per (slot, helicity pair) row (the MIXED mode's
separate tensor-core colour pass, which skips the recomputed events).
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


# (n_g, events, precision name, launch flags): 47 = the lane-group kernel (SIMT colour sums for FP32
# amplitudes, the in-kernel MMA epilogue for MIXED); 63 = MIXED with the separate colour pass
CASES = [(1, 517, "fp32_amp", 39), (2, 1031, "fp32_amp", 47), (2, 1031, "mixed", 47), (2, 1031, "mixed", 63),
         (3, 131, "fp32_amp", 47), (3, 131, "mixed", 63)]


@pytest.mark.parametrize("ng,nevt,prec,flags", CASES)
def test_every_event_recomputed(env, ng, nevt, prec, flags):
    torch, mg, orc = env
    precision = {"fp32_amp": mg.MG_FP32_AMP, "mixed": mg.MG_MIXED}[prec]
    evs, _, _ = orc.events(ng, 70 + ng, nevt)
    with mg.Context(ng) as ctx:
        mom = torch.from_numpy(mg.to_aosoa(evs)).cuda()
        ctx.hel_filter(mom, min(nevt, 1024))
        ref = torch.zeros(nevt, dtype=torch.float64, device="cuda")
        ctx.sigmakin(mom, nevt, ref, mg.MG_FP64)
        ctx.set_launch_shape(precision, 128, 0, flags)
        ctx.set_fp32_tau(1.0)
        got = torch.zeros(nevt, dtype=torch.float64, device="cuda")
        ctx.sigmakin(mom, nevt, got, precision)
        ctx.set_fp32_tau(0.0)        # nothing recomputed: the plain FP32 amplitudes
        plain = torch.zeros(nevt, dtype=torch.float64, device="cuda")
        ctx.sigmakin(mom, nevt, plain, precision)
        assert ctx.check() == 0
    rel = (got / ref - 1).abs()
    assert torch.isfinite(got).all() and rel.max().item() <= 2e-6, rel.max().item()
    # the recomputation did replace the FP32 amplitudes: its error is well below theirs
    rel_plain = (plain / ref - 1).abs()
    assert rel.median().item() < rel_plain.median().item(), (rel.median().item(), rel_plain.median().item())
    # and the oracle agrees on a sample (its own helicity mask from the same warm-up events)
    mask, _ = orc.hel_mask(ng, evs[:min(nevt, 1024)], nthreads=NTHREADS)
    idx = np.arange(0, nevt, max(1, nevt // 16))
    oref = orc.me_batch(ng, evs[idx], mask=mask, nthreads=NTHREADS)
    assert np.max(np.abs(got.cpu().numpy()[idx] / oref - 1)) <= 2e-6
