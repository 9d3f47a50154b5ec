"""mg_sigmakin_noalloc against mg_sigmakin and against the FP64 CPU oracle, through the C ABI.

The no-allocation entry point serves callers that cannot let the library allocate device memory
during a call (a fixed memory budget handed to the engine, or an application pooling allocator
that must stay the only allocator).  It must give the same FP64 matrix elements as the ordinary
entry point, call after call, while its scratch lives in one fixed library array.  This file is
collected last on purpose: the rest of the suite has run when it starts.
"""
import ctypes
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
    import paper_2210_11122_gb300 as mg
    from paper_2210_11122_gb300 import build
    build.build()
    oracle.build()
    return torch, mg, oracle


def _noalloc(L, ctx, mom, nevt, out, stream=None):
    return L.mg_sigmakin_noalloc(ctx._h, ctypes.c_void_p(mom.data_ptr()), nevt, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream) if stream else None)


@pytest.mark.parametrize("proc,nevt", [("ggttg", 65536), ("ggttgg", 3000)])
def test_noalloc_matches_sigmakin_twice(env, proc, nevt):
    torch, mg, _ = env
    L = mg.lib()
    with mg.Context(proc) as ctx:
        stream = torch.cuda.current_stream().cuda_stream
        mom = torch.zeros(ctx.mom_count(nevt), dtype=torch.float64, device="cuda")
        ctx.rambo(11, nevt, 1500.0, mom)
        ref = torch.zeros(nevt, dtype=torch.float64, device="cuda")
        ctx.sigmakin(mom, nevt, ref, mg.MG_FP64)          # also computes the helicity mask
        want = ref.cpu().numpy()
        for _ in range(2):                                 # two calls in a row share the scratch
            got = torch.full((nevt,), -1.0, dtype=torch.float64, device="cuda")
            assert _noalloc(L, ctx, mom, nevt, got, stream) == 0
            g = got.cpu().numpy()
            assert np.max(np.abs(g / want - 1)) <= 1e-12


@pytest.mark.parametrize("ng,nevt", [(0, 203), (1, 131), (2, 67), (3, 37)])
def test_noalloc_matches_oracle(env, ng, nevt):
    """The oracle's own momenta and helicity mask on both sides: every event within 1e-12 of the
    oracle's FP64 matrix element, on two calls in a row."""
    torch, mg, orc = env
    L = mg.lib()
    evs, _, _ = orc.events(ng, 21 + ng, nevt)
    ref_mask, _ = orc.hel_mask(ng, evs, nthreads=NTHREADS)
    ref = orc.me_batch(ng, evs, mask=ref_mask, nthreads=NTHREADS)
    with mg.Context(ng, hel_warmup=nevt) as ctx:
        mom = torch.from_numpy(mg.to_aosoa(evs)).cuda()
        ctx.hel_filter(mom, nevt)
        gmask, _ = ctx.hel_mask()
        assert np.array_equal(gmask, ref_mask)
        for _ in range(2):
            got = torch.full((nevt,), -1.0, dtype=torch.float64, device="cuda")
            assert _noalloc(L, ctx, mom, nevt, got) == 0
            rel = np.abs(got.cpu().numpy() / ref - 1)
            assert rel.max() <= 1e-12, (rel.max(), int(np.argmax(rel)))


def test_noalloc_rejects_oversized_batch_and_missing_mask(env):
    torch, mg, _ = env
    L = mg.lib()
    with mg.Context("ggttggg") as ctx:
        n = 16384 + 32                                     # beyond 2^21 / 128 helicities
        mom = torch.zeros(ctx.mom_count(n), dtype=torch.float64, device="cuda")
        me = torch.zeros(n, dtype=torch.float64, device="cuda")
        # no helicity mask yet
        assert L.mg_sigmakin_noalloc(ctx._h, ctypes.c_void_p(mom.data_ptr()), 64, ctypes.c_void_p(me.data_ptr()),
                                     None) == 1
        ctx.rambo(4, n, 1500.0, mom)
        ctx.hel_filter(mom, 256)
        assert L.mg_sigmakin_noalloc(ctx._h, ctypes.c_void_p(mom.data_ptr()), n, ctypes.c_void_p(me.data_ptr()),
                                     None) == 1
        assert _noalloc(L, ctx, mom, 16384, me) == 0          # the largest batch the scratch holds
        ref = torch.zeros(16384, dtype=torch.float64, device="cuda")
        ctx.sigmakin(mom, 16384, ref, mg.MG_FP64)
        rel = np.abs(me[:16384].cpu().numpy() / ref.cpu().numpy() - 1)
        assert rel.max() <= 1e-12, rel.max()
