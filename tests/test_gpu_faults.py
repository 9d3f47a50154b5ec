"""Faults injected on the host, none on the GPU: an allocation that fails at every allocation site of
context creation, of the first calls of each entry point and of server creation; corrupt and cancelled
serving requests.  Each must return its status (MG_ENOMEM, MG_EINVAL, MG_ECANCELED), leak nothing (the
library's live-allocation count returns to where it was) and leave the library usable, with results
bit-identical to an undisturbed run.
"""
import ctypes
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SQRTS = 1500.0
ENOMEM, EINVAL, ECANCELED = 2, 1, 9


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_11122_gb300 as mg
    from paper_2210_11122_gb300 import build
    build.build()
    yield torch, mg
    mg.diag_fail_alloc(0)


def _fails_with(mg, status, fn):
    with pytest.raises(mg.MGError) as e:
        fn()
    assert e.value.status == status, e.value


def test_context_creation_fails_cleanly_at_every_allocation(env):
    torch, mg = env
    torch.cuda.synchronize()
    base = mg.live_allocs()
    with mg.Context("ggttgg"):
        n = mg.live_allocs() - base
    assert mg.live_allocs() == base and n >= 10
    for k in range(1, n + 1):
        mg.diag_fail_alloc(k)
        _fails_with(mg, ENOMEM, lambda: mg.Context("ggttgg"))
        assert mg.live_allocs() == base, k
    mg.diag_fail_alloc(n + 1)          # one past the last: creation succeeds, the injector stays armed
    with mg.Context("ggttgg"):
        pass
    mg.diag_fail_alloc(0)
    assert mg.live_allocs() == base


def _calls(torch, mg):
    """First calls of each entry point that allocates scratch, on a fresh context: name -> (process,
    function(ctx, mom, n) returning the result as a host array)."""
    def sig(prec):
        def f(ctx, mom, n):
            me = torch.zeros(n, dtype=torch.float64, device="cuda")
            ctx.sigmakin(mom, n, me, prec)
            return me.cpu().numpy()
        return f

    def host(ctx, mom, n):
        me = np.zeros(n)
        ctx.sigmakin_host(mom.cpu().numpy(), n, me, mg.MG_FP64)
        return me

    def lhe(ctx, mom, n):
        me = torch.zeros(n, dtype=torch.float64, device="cuda")
        r = torch.linspace(0.01, 0.99, 2 * n, dtype=torch.float64, device="cuda").reshape(2, n)
        hel = torch.zeros(n, dtype=torch.int32, device="cuda")
        col = torch.zeros(n, dtype=torch.int32, device="cuda")
        ctx.sigmakin_lhe(mom, n, me, r[0].contiguous(), r[1].contiguous(), hel, col, running_alphas=True)
        return np.concatenate([me.cpu().numpy(), hel.cpu().numpy(), col.cpu().numpy()])

    def sde(ctx, mom, n):
        w = torch.zeros(len(mg.sde_channels(ctx.process)) * n, dtype=torch.float64, device="cuda")
        ctx.sde_weights(mom, n, w)
        return w.cpu().numpy()

    return {"fp64": ("ggttg", sig(mg.MG_FP64)), "mixed": ("ggttg", sig(mg.MG_MIXED)),
            "fp64_tccolor": ("ggttgg", sig(mg.MG_FP64_TCCOLOR)), "fp32_amp": ("ggttgg", sig(mg.MG_FP32_AMP)),
            "host": ("ggttg", host), "lhe": ("ggttg", lhe), "sde": ("ggttg", sde)}


@pytest.mark.parametrize("name", ["fp64", "mixed", "fp64_tccolor", "fp32_amp", "host", "lhe", "sde"])
def test_first_call_fails_cleanly_at_every_allocation(env, name):
    torch, mg = env
    proc, fn = _calls(torch, mg)[name]
    n = 777
    with mg.Context(proc) as c0:
        mom = torch.zeros(c0.mom_count(n), dtype=torch.float64, device="cuda")
        c0.rambo(31, n, SQRTS, mom)
    torch.cuda.synchronize()
    base = mg.live_allocs()
    with mg.Context(proc) as ctx:
        before = mg.live_allocs()
        ref = fn(ctx, mom, n)
        m = mg.live_allocs() - before           # allocations of the first call
        assert ctx.check() == 0
    assert m >= 1 and mg.live_allocs() == base
    for k in range(1, m + 1):
        with mg.Context(proc) as ctx:
            mg.diag_fail_alloc(k)
            _fails_with(mg, ENOMEM, lambda: fn(ctx, mom, n))
            mg.diag_fail_alloc(0)
            got = fn(ctx, mom, n)               # the same context, retried: as if nothing had happened
            assert ctx.check() == 0
        assert np.array_equal(got, ref), (name, k)
        assert mg.live_allocs() == base, (name, k)


def test_server_creation_fails_cleanly(env):
    torch, mg = env
    torch.cuda.synchronize()
    base = mg.live_allocs()
    with mg.Server(slots=2, max_nevt=1024):
        n = mg.live_allocs() - base
    assert mg.live_allocs() == base
    ks = sorted(set(list(range(1, 9)) + list(range(9, n + 1, max(1, n // 12))) + [n]))
    for k in ks:
        mg.diag_fail_alloc(k)
        _fails_with(mg, ENOMEM, lambda: mg.Server(slots=2, max_nevt=1024))
        mg.diag_fail_alloc(0)
        assert mg.live_allocs() == base, k


def _alone(torch, mg, proc, seed, nevt):
    """The request computed by hand with the server's resident helicity mask (FP64)."""
    with mg.Context(proc) as ctx:
        warm = torch.zeros(ctx.mom_count(1024), dtype=torch.float64, device="cuda")
        ctx.rambo(mg.SERVE_MASK_SEED, 1024, SQRTS, warm)
        ctx.hel_filter(warm, 1024)
        mom = torch.zeros(ctx.mom_count(nevt), dtype=torch.float64, device="cuda")
        me = torch.zeros(nevt, dtype=torch.float64, device="cuda")
        ctx.rambo_range(seed, 0, nevt, SQRTS, mom)
        ctx.sigmakin(mom, nevt, me, mg.MG_FP64)
        return me.cpu().numpy()


def test_corrupt_and_cancelled_requests(env):
    torch, mg = env
    L = mg.lib()
    torch.cuda.synchronize()
    base = mg.live_allocs()
    chunk = 1024
    with mg.Server(slots=1, max_nevt=chunk, precision=mg.MG_FP64) as srv:
        # corrupt requests are refused at submission and change nothing
        t = ctypes.c_uint64()
        assert L.mg_serve_submit(srv._h, 7, 1, 64, ctypes.byref(t)) == EINVAL
        assert L.mg_serve_submit(srv._h, 0, 1, 0, ctypes.byref(t)) == EINVAL
        assert L.mg_serve_submit(srv._h, 0, 1, -5, ctypes.byref(t)) == EINVAL
        assert L.mg_serve_cancel(srv._h, 987654321) == EINVAL
        # a long request (16 chunks of gg->ttggg, one slot) and one queued behind it
        big = srv.submit("ggttggg", 501, 16 * chunk)
        small = srv.submit("ggtt", 502, 64)
        srv.cancel(small)                        # still queued: nothing of it runs
        time.sleep(0.1)                          # big is in flight by now (a chunk takes ~20 ms)
        srv.cancel(big)                          # in flight: stops at its next chunk boundary
        out = np.full(16 * chunk, -1.0)
        lat = ctypes.c_double()
        assert L.mg_serve_wait(srv._h, big, out.ctypes.data_as(ctypes.c_void_p), 600000, ctypes.byref(lat)) == ECANCELED
        out_s = np.full(64, -1.0)
        assert L.mg_serve_wait(srv._h, small, out_s.ctypes.data_as(ctypes.c_void_p), 600000, ctypes.byref(lat)) == ECANCELED
        assert np.all(out_s == 0.0)
        done = int(np.count_nonzero(out)) // chunk * chunk
        assert 1 <= done // chunk < 16
        assert np.all(out[done:] == 0.0)
        ref = _alone(torch, mg, "ggttggg", 501, done)
        assert np.array_equal(out[:done], ref)
        # the server is still serving, bit-identically
        t2 = srv.submit("ggttg", 503, 3000)
        me, _ = srv.wait(t2)
        assert np.array_equal(me, _alone(torch, mg, "ggttg", 503, 3000))
        st = srv.stats()
        assert st["completed"] == 3 and st["events"] == done + 3000
    assert mg.live_allocs() == base
