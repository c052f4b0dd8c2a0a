"""Profiling driver: the 128^3 bench workload (L = 256 Mpc/h, mesh 256^3, FP32,
DZS merge level 3, seed 2) run from the ICs through `--skip` steps, then
`--steps` more.  Prints "<kernel launches before the profiled steps> <kernel
launches in them>" (the library's own count), so that an ncu command can skip
exactly to the profiled steps:

    read X N <<< $(python -m paper_2005_05328_gb300.profile_run --skip 40 --steps 3)
    ncu --metrics gpu__time_duration.sum --clock-control none -s $X -c $N --csv \\
        --log-file launches.csv python -m paper_2005_05328_gb300.profile_run --skip 40 --steps 3
"""
import argparse

import paper_2005_05328_gb300 as dzs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--skip", type=int, default=40)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--n1d", type=int, default=128)
    a = ap.parse_args()
    dzs.load()
    kw = dict(n1d=a.n1d, mesh=2 * a.n1d, box=2.0 * a.n1d, merge_level=3, seed=2, sigma8=0.8, precision=dzs.FP32)
    with dzs.Context(**kw) as ctx:
        ctx.ics()
        ctx.step(a.skip)
        n0 = int(ctx.counters()[4])
        ctx.step(a.steps)
        n1 = int(ctx.counters()[4])
    print(n0, n1 - n0)


if __name__ == "__main__":
    main()
