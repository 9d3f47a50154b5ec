"""Serving loop (continuous batching) on the GPU through the C ABI.

Each request's result must be the same alone and in a concurrent mix (bit-identical in FP64: the
server's helicity masks are resident, one per process, and every sum has a fixed order),
admission must respect the device-memory cap, and waits are bounded.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SQRTS = 1500.0


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_11122_gb300 as mg
    from paper_2210_11122_gb300 import build
    build.build()
    return torch, mg


def alone(torch, mg, proc, seed, nevt, precision):
    """The request computed by hand with the server's resident helicity mask (the filter on the first
    1,024 events of Philox seed SERVE_MASK_SEED)."""
    with mg.Context(proc) as ctx:
        warm = torch.zeros(ctx.mom_count(1024), dtype=torch.float64, device="cuda")
        ctx.rambo(mg.SERVE_MASK_SEED, 1024, SQRTS, warm)
        ctx.hel_filter(warm, 1024)
        mom = torch.zeros(ctx.mom_count(nevt), dtype=torch.float64, device="cuda")
        me = torch.zeros(nevt, dtype=torch.float64, device="cuda")
        ctx.rambo_range(seed, 0, nevt, SQRTS, mom)
        ctx.sigmakin(mom, nevt, me, precision)
        return me.cpu().numpy()


def mix():
    rng = np.random.default_rng(7)
    out = []
    for r in range(40):
        proc = int(rng.choice(4, p=[0.4, 0.3, 0.2, 0.1]))
        nevt = int(np.exp(rng.uniform(np.log(32), np.log(4096 if proc < 3 else 512))))
        out.append((proc, 1000 + r, nevt))
    return out


@pytest.mark.parametrize("precision", [0, 3])
def test_same_result_alone_and_in_the_mix(env, precision):
    torch, mg = env
    reqs = mix()
    with mg.Server(slots=8, max_nevt=2048, precision=precision) as srv:
        tickets = [srv.submit(p, s, n) for p, s, n in reqs]
        results = [srv.wait(t)[0] for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["peak_inflight"] > 1
    for (p, s, n), got in zip(reqs, results):
        ref = alone(torch, mg, p, s, n, precision)
        assert np.array_equal(got, ref), (p, s, n)


def test_one_slot_equals_many_slots(env):
    torch, mg = env
    reqs = mix()[:16]
    res = {}
    for slots in (1, 6):
        with mg.Server(slots=slots) as srv:
            ts = [srv.submit(p, s, n) for p, s, n in reqs]
            res[slots] = [srv.wait(t)[0] for t in ts]
    for a, b in zip(res[1], res[6]):
        assert np.array_equal(a, b)


def test_admission_respects_memory_cap(env):
    torch, mg = env
    cap = mg.serve_footprint("ggttgg", 2048, mg.MG_FP64)          # room for one such request at a time
    with mg.Server(slots=4, max_nevt=2048, hbm_cap_bytes=cap) as srv:
        ts = [srv.submit("ggttgg", 50 + i, 2048) for i in range(6)]
        for t in ts:
            srv.wait(t)
        st = srv.stats()
    assert st["peak_inflight"] == 1 and st["peak_bytes"] <= cap


def test_bounded_wait_and_chunked_request(env):
    torch, mg = env
    with mg.Server(slots=2, max_nevt=4096) as srv:
        big = srv.submit("ggttggg", 3, 3 * 4096 + 100)               # three full chunks + a ragged one
        with pytest.raises(mg.MGError) as ei:
            srv.wait(big, timeout_ms=1)
        assert ei.value.status == 6                                   # MG_ETIMEOUT, request kept
        me, lat = srv.wait(big)
        assert lat > 0 and np.all(np.isfinite(me)) and np.all(me > 0)
    ref = alone(torch, mg, "ggttggg", 3, 3 * 4096 + 100, mg.MG_FP64)
    assert np.array_equal(me, ref)


def test_served_results_match_oracle(env):
    torch, mg = env
    import oracle
    with mg.Server(slots=3) as srv:
        t = srv.submit("ggtt", 77, 333)
        me, _ = srv.wait(t)
    mom, _, _ = oracle.events(0, 77, 333)
    warm, _, _ = oracle.events(0, mg.SERVE_MASK_SEED, 1024)     # the server's warm-up sample
    mask, _ = oracle.hel_mask(0, warm)
    ref = oracle.me_batch(0, mom, mask=mask)
    assert np.max(np.abs(me / ref - 1)) <= 1e-12


def test_server_masks_are_resident(env):
    """The server computes each process's helicity mask once, at creation: a request of one event gets
    the same mask as a request of thousands (no per-request filter), and its result equals the one
    computed by hand with that mask."""
    torch, mg = env
    with mg.Server(slots=2) as srv:
        one = srv.wait(srv.submit("ggtt", 5, 1))[0]
        many = srv.wait(srv.submit("ggtt", 5, 2048))[0]
    assert one[0] == many[0]
    assert np.array_equal(one, alone(torch, mg, "ggtt", 5, 1, mg.MG_FP64))

