#!/usr/bin/env python
"""Throughput benchmark: matrix elements per second on one or more GB300s.

Metric (the paper's N_events / t_MEs, arXiv 2210.11122 Sec. 2, Tables 1-2): MEs/s of the whole
random numbers -> momenta -> ME path.  One step = one pass of every stage over one batch:
Philox4x32-10 + massive RAMBO (mg_rambo_range), the helicity filter on the batch's first 1,024
events (mg_hel_filter), and the FP64 matrix elements of every event (mg_sigmakin).

Default workload: g g -> t tbar g, 524,288 events per GPU, sqrt(s) = 1500 GeV, m_t = 173 GeV,
alpha_s = 0.118, Philox seed 2.  Under torchrun every rank processes its own disjoint range of
the seed's event stream (weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--process ggttg] [--impl ours|reference]

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "ggtt": dict(ng=0, nevt=16384, seed=1),
    "ggttg": dict(ng=1, nevt=524288, seed=2),
    "ggttgg": dict(ng=2, nevt=262144, seed=3),
    "ggttggg": dict(ng=3, nevt=65536, seed=4),
}
LABEL = {"ggtt": "gg->ttbar", "ggttg": "gg->ttbar g", "ggttgg": "gg->ttbar gg", "ggttggg": "gg->ttbar ggg"}
SQRTS, MT, ALPHAS = 1500.0, 173.0, 0.118
L2_FLUSH_BYTES = 256 << 20
METRIC = "MEs/s"


# ------------------------------------------------------------------------------------------
# multi-rank bookkeeping (one process per GPU; weak scaling, no collective on the data path)
# ------------------------------------------------------------------------------------------
def rank_first_event(rank, nevt_per_rank):
    """Ranks take consecutive disjoint ranges of the seed's event stream: rank r processes events
    [r nevt, (r + 1) nevt), so N ranks reproduce the single-GPU sample of N nevt events."""
    return rank * nevt_per_rank


def max_over_ranks(values, world, device="cpu"):
    """Element-wise maximum over the ranks (the slowest rank sets a step's time)."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def aggregate_rate(world, nevt_per_rank, ms):
    """Whole-job MEs/s: the events of all ranks over the slowest rank's time per step."""
    return world * nevt_per_rank / (ms * 1e-3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--process", default="ggttg", choices=sorted(WORKLOADS))
    ap.add_argument("--nevt", type=int, default=0, help="events per GPU (default: the workload's)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape (fixed launch order)")
    ap.add_argument("--serve", action="store_true", help="serving workload: request trace, p50/p99 latency")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--serve-precision", default="fp64",
                    help="precision of the served form: fp64, fp32_amp, fp64_tccolor or mixed; a comma-separated "
                         "list serves each in turn against one one-at-a-time FP64 baseline")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--no-processes", action="store_true", help="time the configured process only")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg of the default run")
    ap.add_argument("--batch-requests", type=int, default=48,
                    help="jobs of the default run's graph-batch leg (the first requests of the serving trace)")
    ap.add_argument("--serve-requests", type=int, default=500,
                    help="requests of the default run's serving leg (the first ones of the 20,000-request trace)")
    return ap.parse_args()


# sources of the FP64 slot kernels (body, algebra, dispatch): a committed traffic figure holds while their hash does
ME_SOURCES = ("mg_me_kernel.cuh", "mg_me_algebra.cuh", "mg_me2.cu")


def profiled_traffic(kernel_files, profile_md, nevt):
    """DRAM bytes of one launch scaled from a committed ncu summary, or None when the kernel sources
    (hashed in the order given) have changed since the counters were taken."""
    import hashlib
    try:
        h = hashlib.sha256()
        for f in kernel_files:
            h.update(open(f, "rb").read())
        sha = h.hexdigest()[:16]
        fields = {}
        for line in open(profile_md):
            if ":" in line and line.split(":")[0].strip() in ("source_sha256_16", "traffic_bytes_per_event"):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.split()[0]
        if fields.get("source_sha256_16") != sha:
            return None
        return float(fields["traffic_bytes_per_event"]) * nevt
    except (OSError, KeyError, ValueError):
        return None


def config_of(args, nevt, extra=None):
    w = WORKLOADS[args.process]
    c = {"workload": "%s LO QCD, %d events/GPU, sqrt(s)=1500 GeV, m_t=173 GeV, alpha_s=0.118, Philox seed %d"
                     % (LABEL[args.process], nevt, w["seed"]),
         "process": args.process, "events_per_gpu": nevt, "seed": w["seed"],
         "step": "philox+rambo -> helicity filter (1024 warm-up events) -> FP64 matrix elements",
         "l2": "256 MB memset between timed steps, outside the per-step CUDA events",
         "parallelism": "dp%d (disjoint event ranges)" % args.gpus}
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------
def nvsmi_gpu_id(props):
    """nvidia-smi's -i argument for a torch device: its UUID ("GPU-<uuid>").  nvidia-smi ignores
    CUDA_VISIBLE_DEVICES and numbers the GPUs physically, so a visible-device index could name another
    GPU of the machine; the UUID names this one.  None when torch gives no UUID."""
    u = getattr(props, "uuid", None)
    if u is None:
        return None
    u = str(u).strip()
    if not u:
        return None
    return u if u.startswith("GPU-") else "GPU-" + u


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.index = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "gpu": self.index}


# ------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ------------------------------------------------------------------------------------------
def rejected_clocks(clk):
    """A timed region whose clock record disqualifies it: a hardware or thermal slowdown was active, or
    the SM clock sat well below its maximum with no reason given (a leftover clock lock).  A power cap
    alone is kept (and shows in the record)."""
    if not clk:
        return False
    if set(clk.get("reasons") or []) & {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}:
        return True
    sm, mx = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    return bool(sm and mx and sm < 0.8 * mx and not clk.get("reasons"))


def oracle_rate(ng, seed, nevt, target_s=15.0):
    """Events/s of the FP64 oracle's ME on all host cores, over a bounded sample of the workload."""
    import oracle
    cores = os.cpu_count() or 1
    probe = 200 if ng < 2 else (40 if ng == 2 else 8)
    mom, _, _ = oracle.events(ng, seed, probe * cores)
    t = time.perf_counter()
    oracle.me_batch(ng, mom, nthreads=cores)
    rate = probe * cores / (time.perf_counter() - t)
    n = int(max(cores, min(nevt, rate * target_s)))
    mom, _, _ = oracle.events(ng, seed, n)
    t = time.perf_counter()
    oracle.me_batch(ng, mom, nthreads=cores)
    dt = time.perf_counter() - t
    return n / dt, cores, n, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = WORKLOADS[args.process]
    nevt = args.nevt or w["nevt"]
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    # each step: a bounded sample of the workload, sized so the whole run stays within minutes
    _, _, nsamp, dt = oracle_rate(w["ng"], w["seed"], nevt, target_s=min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    mom, _, _ = oracle.events(w["ng"], w["seed"], nsamp)
    for _ in range(args.warmup):
        oracle.me_batch(w["ng"], mom[: max(1, nsamp // 8)], nthreads=cores)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.me_batch(w["ng"], mom, nthreads=cores)
        times.append(time.perf_counter() - t)
    ms = 1e3 * statistics.mean(times)
    value = nsamp / (ms * 1e-3)
    sample = "first %d events of the workload's Philox stream per step (of %d), ME only" % (nsamp, nevt)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MEs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, nevt), "reference": "FP64 CPU oracle (oracle/me_oracle.cpp) on the host cores",
            "cpu_baseline": {"value": value, "unit": "MEs/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "MEs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------------------
# roofline inputs
# ------------------------------------------------------------------------------------------
MODES = (("fp64", 0), ("fp32_amp", 1), ("fp64_tccolor", 2), ("mixed", 3))
# timed steps of a process leg at most (a five-gluon FP64 step takes about a second)
LEG_STEPS = {"ggtt": 20, "ggttg": 20, "ggttgg": 5, "ggttggg": 3}
# events of the autotuner's probe batch per process
TUNE_EVENTS = {"ggtt": 16384, "ggttg": 65536, "ggttgg": 65536, "ggttggg": 8192}
ORACLE_FLOPS = os.path.join(ROOT, "tests", "golden", "oracle_flops.txt")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_TC_TFLOPS = 1900.0


def oracle_flops_table(path=ORACLE_FLOPS):
    """{process: (good helicities, flops per event)} of the FP64 oracle's instrumented count, as stored
    by tests/golden/make_oracle_flops.py (a script that calls only the oracle)."""
    out = {}
    try:
        for line in open(path):
            if line.strip() and not line.startswith("#"):
                f = line.split()
                out[f[0]] = (int(f[2]), int(f[9]))
    except OSError:
        pass
    return out


def tensor_peak(path=PEAKS_FILE):
    """Dense FP16 (FP32 accumulate) tensor-core rate in flop/s and where it comes from: the measured bf16
    burst rate of the GB300s (FP16 and bf16 have the same nominal dense rate), else the fallback."""
    try:
        v = float(json.load(open(path))["bf16_tflops"])
        return v * 1e12, "measured bf16 cuBLAS burst (MEASURED_PEAKS.json) x 1 (nominal f16/bf16 ratio)"
    except (OSError, KeyError, ValueError, TypeError):
        return FALLBACK_TC_TFLOPS * 1e12, "fallback 1.9 PFLOP/s bf16 burst x 1 (nominal f16/bf16 ratio)"


def colour_tc_flops(ncol, good):
    """Tensor-core work of the split-FP16 colour sum per event: for each good helicity the real and
    imaginary jamp rows, each as a hi and a lo FP16 row, times the ncol x ncol matrix (2 ncol^2 flops)."""
    return good * 2 * 2 * 2 * ncol * ncol


def time_roofline(parts, me_ms):
    """Time-based roofline of a kernel mix: T_min = sum over parts of flops / peak (each on its own
    pipe); frac = T_min / measured time."""
    tmin = sum(f / pk for _, f, pk, _ in parts)
    return {"bound": "time", "t_min_ms": tmin * 1e3, "t_ms": me_ms, "frac": tmin / (me_ms * 1e-3),
            "parts": [{"pipe": n, "flops_per_call": f, "peak_tflops": pk / 1e12, "peak_source": src}
                      for n, f, pk, src in parts]}


def fp64_roofline(model_flops, oracle_flops, nevt, me_ms, peak, traffic, kernel):
    """ALU roofline of the FP64 path on the FP64 pipe.  achieved counts the flops of the engine's own
    algorithm (its flop model, pinned to the hardware's FP64 instruction counts); the oracle-count
    figures count the FP64 oracle's instrumented operations (plain recursion per helicity) for the same
    events in the same time, and count_ratio = oracle / engine flops per event."""
    ach = model_flops * nevt / (me_ms * 1e-3)
    r = {"bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s", "frac": ach / peak,
         "traffic": traffic, "kernel": kernel, "flops_per_event": model_flops,
         "peak_source": "measured FP64 DFMA-chain microbenchmark (mg_measure_fma_peak) on this GPU"}
    if oracle_flops:
        ach_o = oracle_flops * nevt / (me_ms * 1e-3)
        r.update({"oracle_flops_per_event": oracle_flops, "oracle_count_achieved": ach_o / 1e12,
                  "oracle_count_frac": ach_o / peak, "count_ratio": oracle_flops / model_flops})
    return r


def profile_for(process):
    """The committed ncu summary of the FP64 matrix-element kernel of a process, if any."""
    import glob
    c = sorted(glob.glob(os.path.join(ROOT, "profiles", "k_me_gluonhel_fp64_%s_*.md" % process)))
    return c[0] if c else None


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
class Leg:
    """One process at its workload size on this rank's GPU: context, momenta and ME buffers, the step
    (Philox + RAMBO -> helicity filter on the first 1,024 events -> matrix elements) and its timing."""

    def __init__(self, mg, torch, process, nevt, rank, stream, flush, autotune):
        w = WORKLOADS[process]
        self.mg, self.torch, self.process, self.nevt = mg, torch, process, nevt
        self.ng, self.seed = w["ng"], w["seed"]
        self.e0 = rank_first_event(rank, nevt)
        self.stream, self.flush = stream, flush
        self.ctx = mg.Context(self.ng, mt=MT, alphas=ALPHAS)
        self.mom = torch.zeros(self.ctx.mom_count(nevt), dtype=torch.float64, device="cuda")
        self.me = torch.zeros(nevt, dtype=torch.float64, device="cuda")
        self.me_x = torch.zeros(nevt, dtype=torch.float64, device="cuda")
        self.nwarm = min(nevt, 1024)
        self.shapes = {}
        self.ctx.rambo_range(self.seed, self.e0, nevt, SQRTS, self.mom, stream=stream)
        if self.ctx.check(stream) != 0:
            raise RuntimeError("RAMBO did not converge")
        if autotune:   # launch shape of the matrix-element kernel per precision (setup, untimed)
            for name, prec in MODES:
                self.ctx.autotune(prec, nevt=min(nevt, TUNE_EVENTS[process]))
        for name, prec in MODES:
            tev, slm, fl = self.ctx.launch_shape(prec)
            self.shapes[name] = {"tile_ev": tev, "slot_major": slm, "flags": fl,
                                 "unrolled": bool(fl & mg.LAUNCH_UNROLLED), "df_redo": bool(fl & mg.LAUNCH_DF_REDO),
                                 "fused": bool(fl & mg.LAUNCH_FUSED), "warp": bool(fl & mg.LAUNCH_WARP),
                                 "tc_apart": bool(fl & mg.LAUNCH_TC_APART), "shared": bool(fl & mg.LAUNCH_SHARED)}

    def step(self, precision, ev):
        ev[0].record(self.stream)
        self.ctx.rambo_range(self.seed, self.e0, self.nevt, SQRTS, self.mom, stream=self.stream)
        self.ctx.hel_filter(self.mom, self.nwarm, stream=self.stream)
        ev[1].record(self.stream)
        self.ctx.sigmakin(self.mom, self.nevt, self.me if precision == self.mg.MG_FP64 else self.me_x, precision,
                          stream=self.stream)
        ev[2].record(self.stream)

    def timed(self, precision, steps, warmup, world):
        """Mean step and matrix-element times (CUDA events on the launching stream, L2 flushed between
        steps outside the events), wall time of the timed region, and the library's kernel launches in it."""
        torch, dist = self.torch, None
        if world > 1:
            import torch.distributed as dist
        mk = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        evs = [mk() for _ in range(steps)]
        with torch.cuda.stream(self.stream):
            for _ in range(warmup):
                self.step(precision, mk())
                self.flush.zero_()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n0 = self.mg.kernel_launches()
        with torch.cuda.stream(self.stream):
            for k in range(steps):
                self.step(precision, evs[k])
                self.flush.zero_()
        nlaunch = self.mg.kernel_launches() - n0
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        wall = time.perf_counter() - t0
        return (statistics.mean(e[0].elapsed_time(e[2]) for e in evs),
                statistics.mean(e[1].elapsed_time(e[2]) for e in evs), wall, nlaunch)

    def rel_err(self):
        rel = ((self.me_x / self.me) - 1).abs().cpu()
        return {"max": float(rel.max()), "p99": float(rel.quantile(0.99) if rel.numel() <= 1 << 24 else rel.max()),
                "median": float(rel.median())}

    def rooflines(self, name, precision, me_ms, peaks, oracle_flops, world):
        """FP64 path: the ALU roofline on the FP64 pipe (engine count, with the oracle-count figures).
        The other modes: the time-based roofline over the pipes their parts run on."""
        mg = self.mg
        mask, ngood = self.ctx.hel_mask()
        flags = self.shapes[name]["flags"]
        amp, col = mg.flops_per_event(self.ng, mask, precision, flags)
        nev = self.nevt
        p64, p32, (ptc, tc_src) = peaks
        src64 = "measured FP64 DFMA-chain microbenchmark (mg_measure_fma_peak)"
        src32 = "measured FP32 FFMA-chain microbenchmark (mg_measure_fma_peak)"
        ncol = math.factorial(self.ng + 2)
        if precision == mg.MG_FP64:
            csrc = os.path.join(ROOT, "paper_2210_11122_gb300", "csrc")
            prof = profile_for(self.process)
            traffic = profiled_traffic([os.path.join(csrc, f) for f in ME_SOURCES], prof, nev) if prof else None
            shared = self.shapes[name]["shared"]
            K = self.ng + 2
            slot_kernel = ("k_me_gluonhel_occ<%d>" % K) if (K >= 4 or (K == 3 and shared)) else ("k_me_gluonhel<%d,double>" % K)
            kernel = ("k_event_prep + %s%s + k_hel_sum (one mg_sigmakin call)"
                      % ("k_share_level (per sequence length) + k_prefix_level (per prefix length) + " if shared else "", slot_kernel))
            return fp64_roofline(amp + col, oracle_flops, nev, me_ms, p64, traffic, kernel)
        if precision == mg.MG_FP64_TCCOLOR:
            return time_roofline([("fp64", amp * nev, p64, src64),
                                  ("tensor_f16", colour_tc_flops(ncol, ngood) * nev, ptc, tc_src)], me_ms)
        # FP32 amplitudes: the per-event FP64 record is the amplitude count with no good helicity
        rec64, _ = mg.flops_per_event(self.ng, [0] * len(mask), precision, flags)
        if precision == mg.MG_FP32_AMP:
            return time_roofline([("fp32", (amp - rec64 + col) * nev, p32, src32), ("fp64", rec64 * nev, p64, src64)],
                                 me_ms)
        return time_roofline([("fp32", (amp - rec64) * nev, p32, src32), ("fp64", rec64 * nev, p64, src64),
                              ("tensor_f16", colour_tc_flops(ncol, ngood) * nev, ptc, tc_src)], me_ms)

    def close(self):
        self.ctx.close()


def epilogue_leg(leg, reps=2):
    """Event-level epilogues on the leg's momenta (one call = all events; CUDA events): FP64 matrix elements
    with the per-event helicity and colour choices and the running coupling (mg_sigmakin_lhe), and the
    single-diagram-enhancement weights of every channel (mg_sde_weights), beside plain FP64 mg_sigmakin."""
    torch, mg = leg.torch, leg.mg
    n = leg.nevt
    gen = torch.Generator(device="cuda").manual_seed(12345)
    rh = torch.rand(n, dtype=torch.float64, device="cuda", generator=gen)
    rc = torch.rand(n, dtype=torch.float64, device="cuda", generator=gen)
    hel = torch.zeros(n, dtype=torch.int32, device="cuda")
    col = torch.zeros(n, dtype=torch.int32, device="cuda")
    nch = len(mg.sde_channels(leg.ng))
    w = torch.zeros(nch * n, dtype=torch.float64, device="cuda")

    def t(fn):
        with torch.cuda.stream(leg.stream):
            fn()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(leg.stream)
            for _ in range(reps):
                fn()
            ev[1].record(leg.stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / reps

    lhe = t(lambda: leg.ctx.sigmakin_lhe(leg.mom, n, leg.me_x, rh, rc, hel, col, True, None, stream=leg.stream))
    sde = t(lambda: leg.ctx.sde_weights(leg.mom, n, w, stream=leg.stream))
    return {"lhe_ms": lhe, "lhe_MEs_per_s": n / (lhe * 1e-3), "sde_ms": sde, "sde_events_per_s": n / (sde * 1e-3),
            "sde_channels": nch,
            "what": "mg_sigmakin_lhe (FP64 MEs + helicity and leading-colour choices + one-loop running alpha_s at "
                    "H_T/2) and mg_sde_weights (single-diagram-enhancement weights of every channel), one call "
                    "over the workload's events"}


def measure_leg(leg, steps, warmup, world, peaks, oracle_flops, modes=MODES):
    """Every precision mode of one process: rates of the whole step and of mg_sigmakin alone, the
    per-event error against the FP64 result of the same events, and the rooflines."""
    out = {}
    for name, prec in modes:
        ms, me_ms, wall, nl = leg.timed(prec, steps, warmup, world)
        ms, me_ms = max_over_ranks([ms, me_ms], world, "cuda")
        r = {"value": aggregate_rate(world, leg.nevt, ms), "ms_per_step": ms, "me_kernel_ms": me_ms,
             "value_me_only": aggregate_rate(world, leg.nevt, me_ms), "steps": steps, "launches_per_step": nl / steps,
             "roofline": leg.rooflines(name, prec, me_ms, peaks, oracle_flops, world)}
        if prec != leg.mg.MG_FP64:
            r["rel_err_vs_fp64"] = leg.rel_err()
        out[name] = r
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2210_11122_gb300 import build as mgbuild
    mgbuild.build()
    import paper_2210_11122_gb300 as mg

    nevt = args.nevt or WORKLOADS[args.process]["nevt"]
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    oflops = oracle_flops_table()
    peaks = (mg.measure_fma_peak(fp32=False, iters=2048), mg.measure_fma_peak(fp32=True, iters=2048), tensor_peak())
    try:
        own_mma = mg.measure_mma_peak(16384)
    except mg.MGError as e:
        own_mma = None
        print("note: tensor-core microbenchmark: %s" % e, file=sys.stderr)
    warm = max(3, args.warmup)

    # ---- headline: the configured process, FP64 step, clocks sampled during the timed region ----
    leg = Leg(mg, torch, args.process, nevt, rank, stream, flush, not args.no_autotune)
    gpu_id = nvsmi_gpu_id(torch.cuda.get_device_properties(local)) or str(local)
    clocks = ClockSampler(gpu_id)
    clocks.start()
    ms_step, ms_me, wall, launches = leg.timed(mg.MG_FP64, args.steps, warm, world)
    clk = clocks.stop()
    # measured again, once, if any rank's clock record disqualifies it (decided by all ranks together:
    # the timed region holds barriers); the first record is kept beside the second
    if max_over_ranks([1.0 if rejected_clocks(clk) else 0.0], world, "cuda")[0] > 0:
        first = clk
        clocks = ClockSampler(gpu_id)
        clocks.start()
        ms_step, ms_me, wall, launches = leg.timed(mg.MG_FP64, args.steps, warm, world)
        clk = clocks.stop()
        if clk is not None:
            clk["remeasured_after"] = first
    nbad = leg.ctx.check(stream)
    ms_step, ms_me = max_over_ranks([ms_step, ms_me], world, "cuda")
    value = aggregate_rate(world, nevt, ms_step)
    ref64 = leg.me.clone()
    _, ngood = leg.ctx.hel_mask()
    roofline = leg.rooflines("fp64", mg.MG_FP64, ms_me, peaks, oflops.get(args.process, (0, 0))[1], world)

    # the other arithmetic modes on the same step
    variants = measure_leg(leg, max(3, args.steps // 2), 3, world, peaks, oflops.get(args.process, (0, 0))[1],
                           modes=MODES[1:])
    leg.me.copy_(ref64)

    # the same FP64 step captured once as a CUDA graph and replayed (one launch per step)
    gmom = torch.zeros_like(leg.mom)
    gme = torch.zeros_like(leg.me)
    gctx = mg.Context(leg.ng, mt=MT, alphas=ALPHAS)
    gctx.set_launch_shape(mg.MG_FP64, leg.shapes["fp64"]["tile_ev"], leg.shapes["fp64"]["slot_major"],
                          leg.shapes["fp64"]["flags"])
    graph = mg.GraphBatch([(gctx, leg.seed, leg.e0, nevt, SQRTS, gmom, gme, mg.MG_FP64)])
    gev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    with torch.cuda.stream(stream):
        for _ in range(3):
            graph.launch(stream)
            flush.zero_()
        for k in range(args.steps):
            gev[2 * k].record(stream)
            graph.launch(stream)
            gev[2 * k + 1].record(stream)
            flush.zero_()
    torch.cuda.synchronize()
    graph_ms = statistics.mean(gev[2 * k].elapsed_time(gev[2 * k + 1]) for k in range(args.steps))
    graph_ms = max_over_ranks([graph_ms], world, "cuda")[0]
    graph_same = bool(torch.equal(gme, leg.me))
    graph.close()
    gctx.close()

    # end to end through the host-buffer entry point (pinned momenta in, MEs out, copies timed), FP64
    # and MIXED
    host_mom = leg.mom.cpu().pin_memory()
    host_me = torch.zeros(nevt, dtype=torch.float64).pin_memory()

    def e2e_of(prec, reps):
        for _ in range(2):
            leg.ctx.sigmakin_host(host_mom, nevt, host_me, prec, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            leg.ctx.sigmakin_host(host_mom, nevt, host_me, prec, stream=stream)
        return max_over_ranks([(time.perf_counter() - t0) / reps], world, "cuda")[0]

    e2e_s = e2e_of(mg.MG_FP64, max(3, args.steps // 2))
    e2e_mixed_s = e2e_of(mg.MG_MIXED, max(3, args.steps))
    e2e = {"value": aggregate_rate(world, nevt, e2e_s * 1e3), "unit": "MEs/s", "h2d_bytes_per_step": int(host_mom.numel() * 8),
           "d2h_bytes_per_step": int(nevt * 8),
           "api": "mg_sigmakin_host: pinned AoSoA momenta -> device -> FP64 MEs -> host (chunked, copies overlapped)",
           "mixed": {"value": aggregate_rate(world, nevt, e2e_mixed_s * 1e3), "ms_per_call": e2e_mixed_s * 1e3,
                     "device_me_ms": variants["mixed"]["me_kernel_ms"]}}
    headline = {"fp64": {"value": value, "ms_per_step": ms_step, "me_kernel_ms": ms_me,
                         "value_me_only": aggregate_rate(world, nevt, ms_me), "steps": args.steps,
                         "roofline": roofline}}
    headline.update(variants)
    shapes = leg.shapes
    epi = epilogue_leg(leg)
    leg.close()

    # ---- every other process of the workloads at its own size: FP64 and the three other modes ----
    processes = {args.process: {"events_per_gpu": nevt, "seed": WORKLOADS[args.process]["seed"],
                                "good_helicities": ngood, "modes": headline, "launch_shapes": shapes,
                                "epilogues": epi}}
    if not args.no_processes:
        for p in ("ggtt", "ggttg", "ggttgg", "ggttggg"):
            if p == args.process:
                continue
            n = WORKLOADS[p]["nevt"]
            lg = Leg(mg, torch, p, n, rank, stream, flush, not args.no_autotune)
            steps = min(args.steps, LEG_STEPS[p])
            modes = measure_leg(lg, steps, 3, world, peaks, oflops.get(p, (0, 0))[1])
            _, g = lg.ctx.hel_mask()
            processes[p] = {"events_per_gpu": n, "seed": WORKLOADS[p]["seed"], "good_helicities": g, "modes": modes,
                            "launch_shapes": lg.shapes, "epilogues": epilogue_leg(lg)}
            lg.close()
            torch.cuda.empty_cache()

    # ---- many small jobs of all processes: per-job launches vs graph branches vs one persistent launch ----
    graph_batch = None
    if not args.no_serve and world == 1:
        graph_batch = batch_leg(mg, torch, stream, flush, args.batch_requests)

    # ---- serving: a bounded sample of the request trace, 80 % load (rank 0, one GPU) ----
    serving = None
    if not args.no_serve and world == 1:
        serving = serve_leg(mg, torch, args.serve_requests, args.slots, ["fp64", "mixed"])

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    cpu = None
    if not args.no_cpu_baseline:
        rate, cores, n, dt = oracle_rate(WORKLOADS[args.process]["ng"], WORKLOADS[args.process]["seed"], nevt)
        cpu = {"value": rate, "unit": "MEs/s", "cores": cores, "kind": "oracle",
               "sample": "first %d events of the workload (of %d), FP64 ME only, %.1f s on %d threads"
                         % (n, nevt, dt, cores)}

    line = {"metric": METRIC, "value": value, "unit": "MEs/s", "n_gpus": world, "steps": args.steps,
            "warmup": warm, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, nevt),
            "me_kernel_ms": ms_me, "wall_s": wall, "nonconverged_events": nbad, "good_helicities": ngood,
            "modes": variants, "launch_shapes": shapes, "processes": processes, "serving": serving,
            "graph_batch": graph_batch,
            "graph": {"ms_per_step": graph_ms, "value": aggregate_rate(world, nevt, graph_ms), "same_result": graph_same,
                      "what": "the FP64 step captured as one CUDA graph (mg_graph_create) and replayed"},
            "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
            "peaks": {"fp64_dfma_tflops": peaks[0] / 1e12, "fp32_ffma_tflops": peaks[1] / 1e12,
                      "f16_mma_tflops": own_mma / 1e12 if own_mma else None,
                      "tensor_denominator_tflops": peaks[2][0] / 1e12,
                      "what": "this GPU, measured by the library's microbenchmarks (mg_measure_fma_peak: FMA chains; "
                              "mg_measure_mma_peak: tcgen05.mma kind::f16 M128 N256 K16, exact integer result checked); "
                              "the tensor rooflines divide by the pool's measured bf16 peak (tensor_denominator_tflops)"},
            "gpu_launches": launches}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------------------------
# serving workload
# ------------------------------------------------------------------------------------------
def serve_trace(mg, torch, n):
    """Request r: Philox4x32-10 words of counter {r, 0, 0, 0}, key {0x5E12E, 0} (the engine's own
    generator): process with probabilities 0.4/0.3/0.2/0.1, nevt log-uniform in [32, 65536] rounded
    up to a multiple of 32, seed = r, exponential inter-arrival variate."""
    import numpy as np
    w = torch.zeros(n * 4, dtype=torch.int32, device="cuda")
    mg.philox(0x5E12E, n, 1, w)
    torch.cuda.synchronize()
    u = (w.cpu().numpy().view(np.uint32).reshape(n, 4).astype(np.float64) + 0.5) * 2.0**-32
    proc = np.searchsorted(np.cumsum([0.4, 0.3, 0.2, 0.1]), u[:, 0], side="right").clip(0, 3)
    nevt = np.floor(np.exp(np.log(32) + u[:, 1] * (np.log(65536) - np.log(32)))).astype(np.int64)
    nevt = ((nevt + 31) // 32) * 32
    expo = -np.log(u[:, 2])
    return proc, nevt, expo


def run_trace(mg, srv, proc, nevt, expo, rate):
    """rate None: closed loop (all submitted at t=0); else Poisson arrivals at `rate` requests/s."""
    import numpy as np
    t0 = time.perf_counter()
    tickets = []
    arrival = 0.0
    for r in range(len(proc)):
        if rate:
            arrival += expo[r] / rate
            dt = t0 + arrival - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
        tickets.append(srv.submit(int(proc[r]), r, int(nevt[r])))
    lat = np.array([srv.wait(t)[1] for t in tickets])
    span = time.perf_counter() - t0
    return span, lat


def batch_leg(mg, torch, stream, flush, nreq, reps=3):
    """The first nreq requests of the serving trace as one batch of FP64 jobs (seed = request id), timed
    three ways with CUDA events: one launch sequence per job on one stream (Philox + RAMBO, helicity filter,
    matrix elements), the CUDA graph with every job on its own branch, and the graph whose matrix elements
    all run in one persistent launch (mg_graph_create_ex, MG_GRAPH_PERSISTENT)."""
    proc, nevt, _ = serve_trace(mg, torch, nreq)
    total = int(nevt.sum())

    def make(persistent):
        jobs = []
        for r in range(nreq):
            c = mg.Context(int(proc[r]), mt=MT, alphas=ALPHAS)
            n = int(nevt[r])
            mom = torch.zeros(c.mom_count(n), dtype=torch.float64, device="cuda")
            me = torch.zeros(n, dtype=torch.float64, device="cuda")
            jobs.append((c, r, 0, n, SQRTS, mom, me, mg.MG_FP64))
        return jobs

    def time_it(fn):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        with torch.cuda.stream(stream):
            fn()
            flush.zero_()
            for k in range(reps):
                ev[2 * k].record(stream)
                fn()
                ev[2 * k + 1].record(stream)
                flush.zero_()
        torch.cuda.synchronize()
        return statistics.mean(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(reps))

    counts = [int((proc == p).sum()) for p in range(4)]
    out = {"workload": "first %d requests of the serving trace as one batch of FP64 jobs: %d events; gg->tt, ttg, "
                       "ttgg, ttggg jobs: %s" % (nreq, total, counts), "events": total}
    jobs = make(False)

    def seq():
        for c, seed, e0, n, q, mom, me, prec in jobs:
            c.rambo_range(seed, e0, n, q, mom, stream=stream)
            c.hel_filter(mom, n, stream=stream)
            c.sigmakin(mom, n, me, prec, stream=stream)
    ms = time_it(seq)
    out["one_launch_sequence_per_job"] = {"ms": ms, "MEs_per_s": total / (ms * 1e-3)}
    g = mg.GraphBatch(jobs)
    ms = time_it(lambda: g.launch(stream))
    out["graph_branches"] = {"ms": ms, "MEs_per_s": total / (ms * 1e-3), "nodes": g.nodes()}
    g.close()
    pj = make(True)
    gp = mg.GraphBatch(pj, persistent=True)
    ms = time_it(lambda: gp.launch(stream))
    out["graph_persistent"] = {"ms": ms, "MEs_per_s": total / (ms * 1e-3), "nodes": gp.nodes()}
    gp.close()
    for j in jobs + pj:
        j[0].close()
    out["speedup_persistent_vs_sequence"] = out["graph_persistent"]["MEs_per_s"] / out["one_launch_sequence_per_job"]["MEs_per_s"]
    return out


def serve_leg(mg, torch, nreq, slots, names):
    """Short serving measurement of the default run: the first nreq requests of the trace, each served
    form closed loop (capacity) and at Poisson arrivals of 80 % of that capacity, against one-at-a-time
    FP64 on the same requests."""
    import numpy as np
    table = {"fp64": mg.MG_FP64, "fp32_amp": mg.MG_FP32_AMP, "fp64_tccolor": mg.MG_FP64_TCCOLOR, "mixed": mg.MG_MIXED}
    proc, nevt, expo = serve_trace(mg, torch, nreq)
    total = int(nevt.sum())
    runs = [("served_" + n, slots, table[n]) for n in names] + [("one_at_a_time_fp64", 1, mg.MG_FP64)]
    out = {}
    for label, sl, precision in runs:
        with mg.Server(slots=sl, precision=precision) as srv:
            w = [srv.submit(p, 10**9 + p, 2048) for p in range(4)]       # warm-up
            for t in w:
                srv.wait(t)
            span, _ = run_trace(mg, srv, proc, nevt, expo, None)
            cap = len(proc) / span
            span2, lat = run_trace(mg, srv, proc, nevt, expo, 0.8 * cap)
            out[label] = {"slots": sl, "capacity_req_per_s": cap, "closed_loop_MEs_per_s": total / span,
                          "open_loop_rate_req_per_s": 0.8 * cap, "open_loop_MEs_per_s": total / span2,
                          "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                          "peak": srv.stats()}
    base = out["one_at_a_time_fp64"]["closed_loop_MEs_per_s"]
    for n in names:
        out["served_" + n]["speedup_closed_loop_vs_one_at_a_time_fp64"] = out["served_" + n]["closed_loop_MEs_per_s"] / base
    out["workload"] = ("first %d requests of the serving trace (gg->tt/ttg/ttgg/ttggg with p=0.4/0.3/0.2/0.1, nevt "
                       "log-uniform in [32, 65536], seed = request id), %d events; Poisson arrivals at 80%% of each "
                       "form's measured capacity; HBM admission cap 64 GiB" % (nreq, total))
    return out


def run_serve(args):
    import numpy as np
    import torch
    from paper_2210_11122_gb300 import build as mgbuild
    mgbuild.build()
    import paper_2210_11122_gb300 as mg
    names = [x.strip() for x in args.serve_precision.split(",") if x.strip()]
    table = {"fp64": mg.MG_FP64, "fp32_amp": mg.MG_FP32_AMP, "fp64_tccolor": mg.MG_FP64_TCCOLOR, "mixed": mg.MG_MIXED}
    for n in names:
        if n not in table:
            raise SystemExit("unknown --serve-precision %r" % n)
    proc, nevt, expo = serve_trace(mg, torch, args.requests)
    total = int(nevt.sum())
    runs = [("served_" + n, args.slots, table[n]) for n in names] + [("one_at_a_time_fp64", 1, mg.MG_FP64)]
    out = {}
    for label, slots, precision in runs:
        with mg.Server(slots=slots, precision=precision) as srv:
            w = [srv.submit(p, 10**9 + p, 2048) for p in range(4)]       # warm-up
            for t in w:
                srv.wait(t)
            span, _ = run_trace(mg, srv, proc, nevt, expo, None)
            cap = len(proc) / span
            span2, lat = run_trace(mg, srv, proc, nevt, expo, 0.8 * cap)
            out[label] = {"slots": slots, "capacity_req_per_s": cap, "closed_loop_MEs_per_s": total / span,
                          "open_loop_rate_req_per_s": 0.8 * cap, "open_loop_MEs_per_s": total / span2,
                          "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                          "peak": srv.stats()}
    s, o = out["served_" + names[0]], out["one_at_a_time_fp64"]
    line = {"metric": "served MEs/s (closed loop) and p50/p99 latency at 80% of capacity", "value":
            s["closed_loop_MEs_per_s"], "unit": "MEs/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": names[0], "data": "synthetic",
            "config": {"workload": "serving mix: %d requests, gg->tt/ttg/ttgg/ttggg with p=0.4/0.3/0.2/0.1, nevt "
                                   "log-uniform in [32, 65536] (multiple of 32), seed = request id, Poisson "
                                   "arrivals at 80%% of measured capacity, HBM admission cap 64 GiB" % args.requests,
                       "requests": args.requests, "events": total},
            "served": s, "one_at_a_time_fp64": o,
            "speedup_closed_loop": s["closed_loop_MEs_per_s"] / o["closed_loop_MEs_per_s"]}
    if len(names) > 1:
        line["served_modes"] = {n: dict(out["served_" + n], speedup_closed_loop=out["served_" + n]["closed_loop_MEs_per_s"]
                                                                           / o["closed_loop_MEs_per_s"]) for n in names}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.serve:
        return run_serve(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
