"""The engine's flop model (mg_flops_per_event_shape, the numerator of bench.py's rooflines) against the
floating-point instructions the GPU executed, as committed in profiles/flops_sigmakin_8192.md (ncu counts
of one mg_sigmakin call of 8,192 events per process and precision, default launch shapes).  No GPU needed.

Tolerances (stated from the captured counts, not tuned after a failure):
  * FP64 path, all kernels of the call: model within 6 % of 2 DFMA + DADD + DMUL per event;
  * FP32 lane-group kernel (4 and 5 gluons): within 6 % of the FP32 flops of the kernel;
  * FP32 kernels with the recursion unrolled at compile time (2 and 3 gluons): the model counts the
    algorithm of the run-time-table kernel; the unrolled code executes 13-15 % fewer FP32 instructions
    (the compiler folds the reflection signs and the constant colour-matrix entries into the FMAs and
    merges common products), so the model is an upper bound there, within 20 %;
  * the FP64 per-event record of the FP32 modes (a few hundred flops per event): within 50 %.
"""
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILE = os.path.join(ROOT, "profiles", "flops_sigmakin_8192.md")
NG = {"ggtt": 0, "ggttg": 1, "ggttgg": 2, "ggttggg": 3}


def hw_lines():
    out = {}
    for line in open(PROFILE):
        f = line.split()
        if len(f) == 6 and f[0] == "hw":
            out[(f[1], f[2])] = tuple(float(x) for x in f[3:])
    return out


@pytest.fixture(scope="module")
def env(orc):
    import paper_2210_11122_gb300 as mg
    from paper_2210_11122_gb300 import build
    build.build()
    warm, _, _ = orc.events(0, 1, 1024)
    mask0, _ = orc.hel_mask(0, warm)
    return mg, mask0


def test_profile_has_every_process_and_precision():
    hw = hw_lines()
    assert set(hw) == {(p, m) for p in NG for m in ("fp64", "fp32_amp")}


@pytest.mark.parametrize("proc", list(NG))
def test_fp64_model_matches_executed_instructions(env, proc):
    mg, mask0 = env
    mask = mask0 if proc == "ggtt" else None
    amp, col = mg.flops_per_event(NG[proc], mask, mg.MG_FP64)
    hw64 = hw_lines()[(proc, "fp64")][0]
    assert abs((amp + col) / hw64 - 1) <= 0.06, (proc, amp + col, hw64)


@pytest.mark.parametrize("proc", list(NG))
def test_fp32_model_matches_executed_instructions(env, proc):
    mg, mask0 = env
    ng = NG[proc]
    mask = mask0 if proc == "ggtt" else None
    nw = ((1 << (ng + 4)) + 31) // 32
    amp, col = mg.flops_per_event(ng, mask, mg.MG_FP32_AMP)
    rec, _ = mg.flops_per_event(ng, [0] * nw, mg.MG_FP32_AMP)
    _, hw32, hwrec = hw_lines()[(proc, "fp32_amp")]
    tol = 0.06 if ng >= 2 else 0.20
    assert abs((amp - rec + col) / hw32 - 1) <= tol, (proc, amp - rec + col, hw32)
    if ng < 2:
        assert amp - rec + col >= hw32          # an upper bound on the unrolled kernels
    assert abs(rec / hwrec - 1) <= 0.5, (proc, rec, hwrec)
