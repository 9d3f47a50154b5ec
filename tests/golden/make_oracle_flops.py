"""Write tests/golden/oracle_flops.txt: the FP64 oracle's operation count per event for each process of
the synthetic workloads (sqrt(s) = 1500 GeV, m_t = 173 GeV, alpha_s = 0.118; seeds 1..4), over the
helicities that the oracle's own filter keeps on the workload's warm-up events (1,024 events; 256 for
five gluons).  Calls only oracle/.

The counter (oracle/me_oracle.cpp) counts every add, subtract and multiply of the plain colour-ordered
recursion, which rebuilds every current and quark-line prefix for every helicity; divisions and square
roots are listed apart and not summed.  These are the "FLOPs per event counted by the instrumented
oracle" of the throughput roofline.

    python tests/golden/make_oracle_flops.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

WORKLOADS = [("ggtt", 0, 1), ("ggttg", 1, 2), ("ggttgg", 2, 3), ("ggttggg", 3, 4)]
OUT = os.path.join(HERE, "oracle_flops.txt")


def rows():
    out = []
    for name, ng, seed in WORKLOADS:
        warm, _, _ = oracle.events(ng, seed, 1024 if ng < 3 else 256)
        mask, _ = oracle.hel_mask(ng, warm, nthreads=os.cpu_count() or 1)
        good = sum(bin(int(w)).count("1") for w in mask)
        c = oracle.flops(ng, warm[0], mask=mask)
        a, col = c["amp"], c["colour"]
        total = a["add"] + a["mul"] + col["add"] + col["mul"]
        out.append((name, ng, good, a["add"], a["mul"], a["div"], a["sqrt"], col["add"], col["mul"], total))
    return out


def main():
    with open(OUT, "w") as f:
        f.write("# FP64 oracle operation counts per event (tests/golden/make_oracle_flops.py): plain colour-ordered\n"
                "# Berends-Giele recursion per good helicity, colour sum C-matrix quadratic form; mask from the\n"
                "# oracle's helicity filter on the workload's warm-up events.  flops = add + mul (amplitudes and\n"
                "# colour); div and sqrt are counted apart.  Event 0 of each workload's seed (divisions depend on\n"
                "# the signs of momentum components; adds and multiplies do not).\n"
                "# columns: process n_g good_helicities amp_add amp_mul amp_div amp_sqrt colour_add colour_mul flops\n")
        for r in rows():
            f.write(" ".join(str(x) for x in r) + "\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()
