"""GPU parity of the event-level epilogues (arXiv 2210.11122 Sec. 4: event-by-event helicities and
leading colours for LHE files; Sec. 2: running alpha_s) through the C ABI, against the FP64 oracle's plain
definitions (oracle/lhe.py) on the oracle's own momenta and helicity mask.

Choices are integers decided by FP64 running sums on both sides; the sums are added in different orders,
so a choice may differ only where the caller's uniform lies within rounding of a boundary -- such an
event is recognised from the oracle's own sums and is the only allowed difference (none is expected).
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
    import oracle.lhe as olhe
    import paper_2210_11122_gb300 as mg
    from paper_2210_11122_gb300 import build
    build.build()
    oracle.build()
    return torch, mg, oracle, olhe


def _near_boundary(weights, r, tol=1e-12):
    tot = float(np.sum(weights))
    cum = np.cumsum(weights)
    return bool(np.any(np.abs(cum - r * tot) <= tol * tot))


def _run_lhe(torch, mg, ctx, mom, n, rh, rc, running):
    me = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    hel = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    col = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    als = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.sigmakin_lhe(mom, n, me, torch.from_numpy(rh).cuda(), torch.from_numpy(rc).cuda(), hel, col, running, als)
    return me.cpu().numpy(), hel.cpu().numpy(), col.cpu().numpy(), als.cpu().numpy()


def _compare(olhe, ng, evs, mask, rh, rc, running, me, hel, col, als, idx=None):
    idx = range(len(evs)) if idx is None else idx
    odd = 0
    for j, i in enumerate(idx):
        rme, rhel, rcol, ra, det = olhe.event(ng, evs[j], mask, r_hel=rh[i], r_col=rc[i], running=running)
        assert abs(me[i] / rme - 1) <= 1e-12, (i, me[i], rme)
        assert abs(als[i] / ra - 1) <= 1e-14, (i, als[i], ra)
        if hel[i] != rhel:
            assert _near_boundary([det["mh"][h] for h in det["good"]], rh[i]), (i, hel[i], rhel)
            odd += 1
        if col[i] != rcol:
            assert _near_boundary(det["w"], rc[i]), (i, col[i], rcol)
            odd += 1
    return odd


@pytest.mark.parametrize("running", [False, True])
@pytest.mark.parametrize("ng,nevt", [(0, 97), (1, 131), (2, 41), (3, 13)])
def test_lhe_epilogue_matches_oracle(env, ng, nevt, running):
    torch, mg, orc, olhe = env
    evs, _, _ = orc.events(ng, 40 + ng, nevt)
    mask, _ = orc.hel_mask(ng, evs, nthreads=NTHREADS)
    rng = np.random.default_rng(100 + ng)
    rh, rc = rng.random(nevt), rng.random(nevt)
    with mg.Context(ng, hel_warmup=nevt) as ctx:
        mom = torch.from_numpy(mg.to_aosoa(evs)).cuda()
        ctx.hel_filter(mom, nevt)
        gmask, _ = ctx.hel_mask()
        assert np.array_equal(gmask, mask)
        me, hel, col, als = _run_lhe(torch, mg, ctx, mom, nevt, rh, rc, running)
        # the plain FP64 entry point agrees with the epilogue's helicity sum (fixed coupling)
        if not running:
            me64 = torch.zeros(nevt, dtype=torch.float64, device="cuda")
            ctx.sigmakin(mom, nevt, me64, mg.MG_FP64)
            assert np.max(np.abs(me / me64.cpu().numpy() - 1)) <= 1e-13
    assert np.all(hel >= 0) and np.all(col >= 0) and np.all(col < orc.ncol(ng))
    for h in hel:
        assert (int(mask[h >> 5]) >> (int(h) & 31)) & 1
    assert _compare(olhe, ng, evs, mask, rh, rc, running, me, hel, col, als) == 0


def test_lhe_epilogue_full_size_sampled(env):
    """gg->ttggg at its full workload size (65,536 events: ten chunks of 6,848 events, the shared-current
    scratch's bound, inside the jamp-square scratch's 34,944): the sampled events, on both sides of chunk
    boundaries, carry the oracle's momenta in the full-size buffer; their MEs, couplings and choices
    match the oracle's."""
    torch, mg, orc, olhe = env
    ng, seed, n = 3, 4, 65536
    npar = ng + 4
    rng = np.random.default_rng(7)
    rh, rc = rng.random(n), rng.random(n)
    idx = np.unique(np.concatenate([[0, 6847, 6848, 34943, 34944, 61631, 61632, n - 1], rng.integers(0, n, 8)]))
    ev = np.concatenate([orc.events(ng, seed, 1, e0=int(i))[0] for i in idx])
    warm, _, _ = orc.events(ng, seed, 256)
    mask, _ = orc.hel_mask(ng, warm, nthreads=NTHREADS)
    with mg.Context(ng) as ctx:
        mom = torch.zeros(ctx.mom_count(n), dtype=torch.float64, device="cuda")
        ctx.rambo(seed, n, SQRTS, mom)
        ctx.hel_filter(mom, 1024)
        gmask, _ = ctx.hel_mask()
        assert np.array_equal(gmask, mask)
        momh = mom.cpu().numpy()
        view = momh.reshape(-1, npar, 4, mg.PAGE)
        for j, e in enumerate(idx):
            view[e // mg.PAGE, :, :, e % mg.PAGE] = ev[j]
        mom.copy_(torch.from_numpy(momh))
        me, hel, col, als = _run_lhe(torch, mg, ctx, mom, n, rh, rc, True)
    assert np.all(np.isfinite(me)) and np.all(me > 0)
    assert _compare(olhe, ng, ev, mask, rh, rc, True, me, hel, col, als, idx=idx) == 0


@pytest.mark.parametrize("prec", [0, 3])
def test_alphas_running_any_mode(env, prec):
    """mg_alphas_running rescales the matrix elements of any mode in place by (alpha_s(H_T/2)/alpha_s)^(n+2);
    the FP64 result equals the oracle evaluated at the running coupling."""
    torch, mg, orc, olhe = env
    ng, n = 1, 333
    evs, _, _ = orc.events(ng, 12, n)
    with mg.Context(ng) as ctx:
        mom = torch.from_numpy(mg.to_aosoa(evs)).cuda()
        me = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.sigmakin(mom, n, me, prec)
        before = me.cpu().numpy()
        als = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.alphas_running(mom, n, me, als)
        after, a = me.cpu().numpy(), als.cpu().numpy()
    ra = np.array([olhe.alphas_1loop(0.118, olhe.half_ht(p, 173.0)) for p in evs])
    assert np.max(np.abs(a / ra - 1)) <= 1e-14
    assert np.max(np.abs(after / before / (ra / 0.118) ** 3 - 1)) <= 1e-14
    if prec == 0:
        mask, _ = orc.hel_mask(ng, evs[:1024], nthreads=NTHREADS)
        ref = np.array([orc.me_batch(ng, evs[i:i + 1], mask=mask, alphas=ra[i])[0] for i in range(n)])
        assert np.max(np.abs(after / ref - 1)) <= 1e-12
