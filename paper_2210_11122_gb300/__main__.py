"""Time one matrix-element configuration on the current GPU:

    python -m paper_2210_11122_gb300 --process ggttg --nevt 524288 --precision fp32_amp [--calls 8]
                                     [--flags N] [--seed 2] [--time-filter]

Draws nevt events (Philox + RAMBO, sqrt(s) = 1500 GeV), runs the helicity filter on the first 1024
(with --time-filter: three more times, timed), then calls mg_sigmakin `calls` times (the first three
untimed) and prints the mean time per call and the MEs/s of one call.  --flags sets the launch flags
(MG_LAUNCH_* of mg.h) instead of the defaults.  Without --time-filter the launch sequence is one
filter, then the mg_sigmakin calls (what the ncu commands of the committed profiles count on).
"""
import argparse
import sys


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2210_11122_gb300")
    ap.add_argument("--process", default="ggttg", choices=["ggtt", "ggttg", "ggttgg", "ggttggg"])
    ap.add_argument("--nevt", type=int, default=524288)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_amp", "fp64_tccolor", "mixed"])
    ap.add_argument("--calls", type=int, default=8)
    ap.add_argument("--flags", type=int, default=None)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--time-filter", action="store_true")
    args = ap.parse_args(argv)

    import torch
    import paper_2210_11122_gb300 as mg
    from paper_2210_11122_gb300 import build
    build.build()
    ng = ["ggtt", "ggttg", "ggttgg", "ggttggg"].index(args.process)
    prec = {"fp64": mg.MG_FP64, "fp32_amp": mg.MG_FP32_AMP, "fp64_tccolor": mg.MG_FP64_TCCOLOR,
            "mixed": mg.MG_MIXED}[args.precision]
    with mg.Context(ng) as ctx:
        if args.flags is not None:
            ctx.set_launch_shape(prec, 128, 0, args.flags)
        mom = torch.zeros(ctx.mom_count(args.nevt), dtype=torch.float64, device="cuda")
        me = torch.zeros(args.nevt, dtype=torch.float64, device="cuda")
        ctx.rambo(args.seed, args.nevt, 1500.0, mom)
        ctx.hel_filter(mom, min(args.nevt, 1024))
        filter_ms = None
        if args.time_filter:
            torch.cuda.synchronize()
            fev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            fev[0].record()
            for _ in range(3):
                ctx.hel_filter(mom, min(args.nevt, 1024))
            fev[1].record()
            torch.cuda.synchronize()
            filter_ms = fev[0].elapsed_time(fev[1]) / 3
        warm = min(3, args.calls)
        for _ in range(warm):
            ctx.sigmakin(mom, args.nevt, me, prec)
        torch.cuda.synchronize()
        timed = args.calls - warm
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(timed):
            ctx.sigmakin(mom, args.nevt, me, prec)
        ev[1].record()
        torch.cuda.synchronize()
        if timed > 0:
            ms = ev[0].elapsed_time(ev[1]) / timed
            print("%s %d events %s: %.4f ms per call, %.4g MEs/s%s"
                  % (args.process, args.nevt, args.precision, ms, args.nevt / (ms * 1e-3),
                     "" if filter_ms is None else "; helicity filter %.4f ms" % filter_ms))
    return 0


if __name__ == "__main__":
    sys.exit(main())
