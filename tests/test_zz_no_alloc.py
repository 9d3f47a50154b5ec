"""mg_sigmakin_noalloc against mg_sigmakin, through the C ABI.

The no-allocation entry point serves callers that cannot let the library allocate device memory
during a call (a fixed memory budget handed to the engine, or an application pooling allocator
that must stay the only allocator).  It must give the same FP64 matrix elements as the ordinary
entry point, call after call, while its scratch lives in one fixed library array.  This file is
collected last on purpose: the rest of the suite has run when it starts.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_11122_gb300 as mg
    from paper_2210_11122_gb300 import build
    build.build()
    return torch, mg


@pytest.mark.parametrize("proc,nevt", [("ggttg", 65536), ("ggttgg", 3000)])
def test_noalloc_matches_sigmakin_twice(env, proc, nevt):
    torch, mg = env
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
            rc = L.mg_sigmakin_noalloc(ctx._h, ctypes.c_void_p(mom.data_ptr()), nevt, ctypes.c_void_p(got.data_ptr()),
                                       ctypes.c_void_p(stream))
            assert rc == 0
            g = got.cpu().numpy()
            assert np.max(np.abs(g / want - 1)) <= 1e-12


def test_noalloc_rejects_oversized_batch_and_missing_mask(env):
    torch, mg = env
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
        assert L.mg_sigmakin_noalloc(ctx._h, ctypes.c_void_p(mom.data_ptr()), 16384, ctypes.c_void_p(me.data_ptr()),
                                     None) == 0
        torch.cuda.synchronize()
