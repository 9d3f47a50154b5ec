"""C ABI checks that need no GPU: the library loads, exports every entry point that
include/mg.h declares, and its host-only logic (colour matrix, sizes, layout, argument
validation) is right.  No compute call is made here."""
import ctypes
import os
import re
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def mg():
    import paper_2210_11122_gb300 as m
    from paper_2210_11122_gb300 import build
    build.build()
    return m


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("mg_create", "mg_destroy", "mg_rambo", "mg_sigmakin", "mg_hel_mask", "mg_philox", "mg_strerror"):
        assert name in syms


def test_binding_constants_match_the_header(mg):
    """The Python binding's enum values and launch flags are the header's."""
    src = open(os.path.join(ROOT, "include", "mg.h")).read()
    flags = dict((k, int(v)) for k, v in re.findall(r"#define MG_LAUNCH_([A-Z_]+)\s+(\d+)", src))
    assert flags and all(getattr(mg, "LAUNCH_" + k) == v for k, v in flags.items())
    enums = dict((k, int(v)) for k, v in re.findall(r"\b(MG_[A-Z0-9_]+)\s*=\s*(\d+)", src))
    for name in ("MG_FP64", "MG_FP32_AMP", "MG_FP64_TCCOLOR", "MG_MIXED", "MG_GG_TT", "MG_GG_TTG", "MG_GG_TTGG",
                 "MG_GG_TTGGG"):
        assert getattr(mg, name) == enums[name], name
    status = {k: v for k, v in enums.items() if k == "MG_OK" or k.startswith("MG_E")}
    assert {v: k for k, v in status.items()} == mg.STATUS


def test_library_exports_every_declared_symbol(mg):
    L = ctypes.CDLL(mg.library_path())
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert not missing, missing


def test_strerror_and_defaults(mg):
    for s in range(10):
        assert mg.lib().mg_strerror(s)
    assert mg.lib().mg_strerror(9) != mg.lib().mg_strerror(99)
    p = mg.default_params()
    assert (p.mt, p.wt, p.alphas, p.hel_warmup, p.hel_tau) == (173.0, 0.0, 0.118, 1024, 1e-9)


def test_process_info(mg):
    for name, (npar, nhel, ncol, nd) in {"ggtt": (4, 16, 2, 3), "ggttg": (5, 32, 6, 16), "ggttgg": (6, 64, 24, 123),
                                         "ggttggg": (7, 128, 120, 1240)}.items():
        assert mg.process_info(name) == {"npar": npar, "nhel": nhel, "ncol": ncol, "ndiagrams": nd}
    with pytest.raises(mg.MGError):
        mg.process_info(7)


def test_mom_count_pads_to_pages(mg):
    assert mg.mom_count("ggtt", 0) == 0
    assert mg.mom_count("ggtt", 1) == 32 * 4 * 4
    assert mg.mom_count("ggttggg", 33) == 64 * 7 * 4
    assert mg.mom_count("ggtt", -1) == -1


@pytest.mark.parametrize("proc,k", [("ggtt", 2), ("ggttg", 3), ("ggttgg", 4), ("ggttggg", 5)])
def test_colour_matrix_matches_oracle(mg, proc, k):
    """The library's U(N)-loop-counting colour matrix equals the oracle's Fierz reduction exactly."""
    from oracle import colour
    num, den = mg.colour_matrix(proc)
    ex = colour.colour_matrix_exact(k)
    n = len(ex)
    assert num.shape == (n, n)
    for a in range(n):
        for b in range(n):
            assert Fraction(int(num[a, b]), den) == ex[a][b]


def test_aosoa_roundtrip(mg):
    rng = np.random.default_rng(0)
    for nevt in (1, 31, 32, 33, 100):
        m = rng.normal(size=(nevt, 5, 4))
        buf = mg.to_aosoa(m)
        assert buf.size == mg.mom_count("ggttg", nevt)
        assert np.array_equal(mg.from_aosoa(buf, nevt, 5), m)
        # element (e, i, mu) at ((e/32) npar + i) 4 32 + mu 32 + e%32
        e, i, mu = nevt - 1, 3, 2
        assert buf[((e // 32) * 5 + i) * 128 + mu * 32 + e % 32] == m[e, i, mu]


def test_flop_model(mg):
    for proc in ("ggtt", "ggttg", "ggttgg", "ggttggg"):
        info = mg.process_info(proc)
        n, nh = info["ncol"], info["nhel"]
        amp, col = mg.flops_per_event(proc)
        assert amp > 0
        assert col == nh * (4.0 * n * (n + 1) / 2 + 4 * n)
        # a mask with fewer good helicities costs less
        mask = np.zeros((nh + 31) // 32, dtype=np.uint32)
        mask[0] = 1
        amp1, col1 = mg.flops_per_event(proc, mask)
        assert col1 == 4.0 * n * (n + 1) / 2 + 4 * n and 0 < amp1 < amp
        # the tensor-core colour mode keeps the FP64 amplitude algorithm; the FP32 modes form (gamma.J) v
        # per jamp term instead of tabulating it, the same colour sums -- except the lane-group kernel
        # (default for 4 and 5 gluons) in MG_FP32_AMP, whose SIMT epilogue multiplies the full colour
        # matrix into all four helicities of a slot (its MG_MIXED colour sums run on the tensor cores)
        assert mg.flops_per_event(proc, None, mg.MG_FP64_TCCOLOR) == (amp, col)
        a32, c32 = mg.flops_per_event(proc, None, mg.MG_FP32_AMP)
        assert a32 != amp
        if info["npar"] < 6:
            assert c32 == col
        else:
            assert c32 == (nh // 4) * 4 * (4.0 * n * n + 4 * n)
        assert mg.flops_per_event(proc, None, mg.MG_MIXED) == (a32, col)
        # FP64 amplitudes with the currents shared between gluon-helicity combinations: fewer flops with
        # every helicity good from 1 final-state gluon on, the same colour sums; the default there;
        # no effect on the FP32-amplitude modes
        sh = mg.flops_per_event(proc, None, mg.MG_FP64, mg.LAUNCH_SHARED)
        plain = mg.flops_per_event(proc, None, mg.MG_FP64, 0)
        assert sh[1] == plain[1] == col
        if proc != "ggtt":
            assert sh[0] < plain[0]
        assert (amp, col) == (sh if proc != "ggtt" else plain)
        warp = mg.LAUNCH_WARP if info["npar"] >= 6 else 0   # the FP32 default for 4 and 5 gluons
        assert mg.flops_per_event(proc, None, mg.MG_FP32_AMP, mg.LAUNCH_SHARED | warp) == (a32, c32)
    with pytest.raises(mg.MGError):
        mg.flops_per_event("ggttg", None, 7)


def test_invalid_arguments_rejected_without_gpu(mg):
    L = mg.lib()
    assert L.mg_rambo(None, 1, 10, 1500.0, None, None, None) == 1
    assert L.mg_sigmakin(None, None, 10, 0, None, None) == 1
    assert L.mg_hel_mask(None, None, None) == 1
    assert L.mg_diag_tc_stall(None, 1) == 1
    assert L.mg_philox(1, -1, 2, None, None) == 1
    assert L.mg_create(9, None, ctypes.byref(ctypes.c_void_p())) == 1
    assert L.mg_create(0, None, None) == 1
    # rejected calls launch nothing: the process-wide launch count does not move
    n0 = mg.kernel_launches()
    assert L.mg_sigmakin(None, None, 10, 0, None, None) == 1
    assert L.mg_philox(1, -1, 2, None, None) == 1
    assert mg.kernel_launches() == n0 >= 0


def test_serve_footprint_host(mg):
    """Admission footprint of a request: momenta + MEs + per-helicity partial sums + per-event records
    (+ FP32 jamps for the tensor-core colour modes)."""
    for proc in ("ggtt", "ggttg", "ggttgg", "ggttggg"):
        info = mg.process_info(proc)
        npar, nhel, ncol = info["npar"], info["nhel"], info["ncol"]
        f64 = mg.serve_footprint(proc, 100, mg.MG_FP64)
        n = 128
        assert f64 > n * (npar * 4 * 8 + 8 + nhel * 8)
        ftc = mg.serve_footprint(proc, 100, mg.MG_FP64_TCCOLOR)
        assert ftc - f64 == n * nhel * ncol * 8
        assert mg.serve_footprint(proc, 1000, mg.MG_FP64) > f64
    assert mg.serve_footprint(9, 10, 0) == -1


def test_colour_flow_is_the_lexicographic_permutation(mg):
    """Colour flow index = lexicographic rank of the gluon ordering along the quark line (the jamp index
    of mg_sigmakin_lhe's colour choice); out-of-range flows are rejected."""
    from itertools import permutations
    for proc, k in (("ggtt", 2), ("ggttg", 3), ("ggttgg", 4), ("ggttggg", 5)):
        for c, perm in enumerate(permutations(range(k))):
            assert mg.colour_flow(proc, c) == list(perm)
        with pytest.raises(mg.MGError):
            mg.colour_flow(proc, len(list(permutations(range(k)))))


def test_sde_channel_keys_equal_the_oracles(mg):
    """The library's single-diagram-enhancement channels (its own enumeration) are the oracle's, key for
    key (3 / 15 / 105 / 945 three-point-vertex diagrams)."""
    from oracle import sde
    for ng, proc in enumerate(("ggtt", "ggttg", "ggttgg", "ggttggg")):
        keys = mg.sde_channels(proc)
        assert len(keys) == len(set(keys)) == [3, 15, 105, 945][ng]
        assert set(keys) == {sde.key(d) for d in sde.diagrams(ng)}


def test_allocation_fault_injector_host(mg):
    """The host-side allocation-failure injector: argument checks and the live count without a GPU."""
    L = mg.lib()
    assert L.mg_diag_fail_alloc(-1) == 1
    assert L.mg_diag_fail_alloc(3) == 0
    assert L.mg_diag_fail_alloc(0) == 0
    assert mg.live_allocs() == 0              # nothing allocated in a process without a device
    assert L.mg_serve_cancel(None, 1) == 1
    r = ctypes.c_double()
    assert L.mg_measure_mma_peak(0, ctypes.byref(r)) == 1 and L.mg_measure_mma_peak(1 << 17, ctypes.byref(r)) == 1
    assert L.mg_measure_mma_peak(16, None) == 1
    assert L.mg_set_fp32_tau(None, ctypes.c_double(1e-4)) == 1
