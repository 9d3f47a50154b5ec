"""Launch-shape autotuner and CUDA-graph batches through the C ABI (GPU)."""
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


def step(torch, mg, ctx, seed, e0, nevt, precision):
    mom = torch.zeros(ctx.mom_count(nevt), dtype=torch.float64, device="cuda")
    me = torch.zeros(nevt, dtype=torch.float64, device="cuda")
    ctx.rambo_range(seed, e0, nevt, SQRTS, mom)
    ctx.hel_filter(mom, nevt)
    ctx.sigmakin(mom, nevt, me, precision)
    return me.cpu().numpy()


@pytest.mark.parametrize("proc,precision", [("ggttg", 0), ("ggttgg", 1), ("ggttggg", 3)])
def test_autotune_keeps_results_and_caches(env, proc, precision, tmp_path):
    torch, mg = env
    cache = str(tmp_path / "shapes.txt")
    with mg.Context(proc) as ctx:
        ref = step(torch, mg, ctx, 5, 0, 1000, precision)
        tev, sm, ms = ctx.autotune(precision, nevt=2048, cache_path=cache)
        assert tev in (32, 64, 128) and sm in (0, 1) and ms > 0
        got = step(torch, mg, ctx, 5, 0, 1000, precision)
    if precision == mg.MG_FP64:
        assert np.array_equal(got, ref)      # FP64: the shape changes scheduling, not arithmetic
    else:
        # FP32 modes: the autotuner also chooses among kernels (other FP32 summation orders); every one
        # stays within 1e-5 of FP64, so two of them agree within 2e-5
        assert np.max(np.abs(got / ref - 1)) <= 2e-5
    line = open(cache).read().split()
    assert int(line[1]) == tev and int(line[2]) == sm
    with mg.Context(proc) as ctx2:           # second context: taken from the cache without timing
        assert ctx2.autotune(precision, nevt=2048, cache_path=cache)[:2] == (tev, sm)


def test_graph_batch_matches_step_by_step(env):
    torch, mg = env
    sizes = {"ggtt": 3000, "ggttg": 2000, "ggttgg": 700, "ggttggg": 96}
    ctxs = {p: mg.Context(p) for p in sizes}
    bufs = {p: (torch.zeros(ctxs[p].mom_count(n), dtype=torch.float64, device="cuda"),
                torch.zeros(n, dtype=torch.float64, device="cuda")) for p, n in sizes.items()}

    def jobs(seed0):
        return [(ctxs[p], seed0 + i, 0, n, SQRTS, bufs[p][0], bufs[p][1], mg.MG_FP64) for i, (p, n) in enumerate(sizes.items())]

    g = mg.GraphBatch(jobs(100))
    assert g.nodes() >= 4 * 5
    for seed0 in (100, 200):
        if seed0 != 100:
            g.update(jobs(seed0))
        g.launch()
        torch.cuda.synchronize()
        got = {p: bufs[p][1].cpu().numpy().copy() for p in sizes}
        for i, (p, n) in enumerate(sizes.items()):
            with mg.Context(p) as c:
                ref = step(torch, mg, c, seed0 + i, 0, n, mg.MG_FP64)
            assert np.array_equal(got[p], ref), p
    g.close()
    for c in ctxs.values():
        c.close()


def test_graph_rejects_shared_context(env):
    torch, mg = env
    with mg.Context("ggttg") as ctx:
        mom = torch.zeros(ctx.mom_count(64), dtype=torch.float64, device="cuda")
        me = torch.zeros(64, dtype=torch.float64, device="cuda")
        j = (ctx, 1, 0, 64, SQRTS, mom, me, mg.MG_FP64)
        with pytest.raises(mg.MGError) as ei:
            mg.GraphBatch([j, j])
        assert ei.value.status == 1


def test_launch_shape_set_and_get(env):
    torch, mg = env[0], env[1]
    with mg.Context(1) as ctx:
        both = mg.LAUNCH_UNROLLED | mg.LAUNCH_DF_REDO | mg.LAUNCH_FUSED | mg.LAUNCH_SHARED
        assert ctx.launch_shape(mg.MG_FP32_AMP) == (128, 0, both)
        ctx.set_launch_shape(mg.MG_FP32_AMP, 32, 1, mg.LAUNCH_DF_REDO)
        assert ctx.launch_shape(mg.MG_FP32_AMP) == (32, 1, mg.LAUNCH_DF_REDO)
        assert ctx.launch_shape(mg.MG_FP64) == (128, 0, both)
        for bad in ((48, 0, 1), (64, 2, 1), (64, 0, 128)):
            with pytest.raises(mg.MGError):
                ctx.set_launch_shape(mg.MG_FP32_AMP, *bad)


@pytest.mark.parametrize("precision", [1, 3])
def test_graph_batch_fp32_modes(env, precision):
    """The FP32-amplitude modes captured into a graph batch -- their FP32 pre-pass, the recomputation
    forked onto each context's side stream and joined back, the tensor-core colour sums -- give the
    same bits as the same steps called one by one."""
    torch, mg = env
    sizes = {"ggtt": 3000, "ggttg": 2000, "ggttgg": 700, "ggttggg": 96}
    ctxs = {p: mg.Context(p) for p in sizes}
    bufs = {p: (torch.zeros(ctxs[p].mom_count(n), dtype=torch.float64, device="cuda"),
                torch.zeros(n, dtype=torch.float64, device="cuda")) for p, n in sizes.items()}
    jobs = [(ctxs[p], 300 + i, 0, n, SQRTS, bufs[p][0], bufs[p][1], precision) for i, (p, n) in enumerate(sizes.items())]
    g = mg.GraphBatch(jobs)
    for _ in range(2):
        g.launch()
    torch.cuda.synchronize()
    got = {p: bufs[p][1].cpu().numpy().copy() for p in sizes}
    for i, (p, n) in enumerate(sizes.items()):
        ref = step(torch, mg, ctxs[p], 300 + i, 0, n, precision)
        assert np.array_equal(got[p], ref), p
    g.close()
    for c in ctxs.values():
        c.close()


def test_kernel_launch_counter(env):
    # mg_kernel_launches brackets the kernels of the calls between two reads: an FP64 gg->ttg call is
    # the per-event record, the matrix elements and the helicity sum, plus, with shared currents, one pass
    # per sequence length (1 and 2 gluons) and one per quark-line prefix length (1 and 2 gluons)
    torch, mg = env
    n = 4096
    with mg.Context("ggttg") as ctx:
        mom = torch.zeros(ctx.mom_count(n), dtype=torch.float64, device="cuda")
        me = torch.zeros(n, dtype=torch.float64, device="cuda")
        c0 = mg.kernel_launches()
        ctx.rambo(2, n, SQRTS, mom)
        assert mg.kernel_launches() > c0
        ctx.hel_filter(mom, 1024)
        counts = {}
        for flags in (mg.LAUNCH_UNROLLED | mg.LAUNCH_FUSED | mg.LAUNCH_SHARED, mg.LAUNCH_UNROLLED | mg.LAUNCH_FUSED):
            ctx.set_launch_shape(mg.MG_FP64, 128, 0, flags)
            c0 = mg.kernel_launches()
            ctx.sigmakin(mom, n, me, mg.MG_FP64)
            counts[flags] = mg.kernel_launches() - c0
        torch.cuda.synchronize()
    assert list(counts.values()) == [7, 3]
