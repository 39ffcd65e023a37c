"""Switching campaign of the paper's GdFeCo protocol (Sec. II.D, II.G) on one
GPU: every (peak T_e, cooling multiplier d, realisation) is an instance of one
batched system; prints the switching probability per (peak, d) with its
Wilson 95 % interval, and the throughput.

    python -m paper_2608_18541_b300.campaign --peaks 800 1100 1400 2000 --ds 2 4 6 8 --reps 8
"""
import argparse
import json
import time

import numpy as np

from . import System
from . import protocol as PR
from . import workloads as W

FS = 1e-15


def run(peaks, ds, reps, n=13, t_peak=500 * FS, t_cool=500 * FS, t_tail=2000 * FS, dt=0.2 * FS, precision=32,
        sweep="symmetric", sample_every=50, stream=None):
    sysd, bath, steps = W.switching_campaign(peaks, ds, reps, n=n, t_peak=t_peak, t_cool=t_cool, t_tail=t_tail,
                                             dt=dt, sample_every=sample_every)
    sysd = dict(sysd, sweep=sweep)
    g = System(sysd, bath, precision=precision, stream=stream,
               obs_capacity=steps // sample_every + 2)
    g.sync()
    t0 = time.perf_counter()
    g.step(steps)
    g.sync()
    secs = time.perf_counter() - t0
    cells = {}
    for k, inst in enumerate(sysd["instances"]):
        rows = g.observables(k)
        cells.setdefault((inst["peak_Te"], round(inst["fwhm"] / t_cool)), []).append(
            PR.gd_switched(rows, t_peak + inst["fwhm"]))
    table = []
    for (T, d), v in sorted(cells.items()):
        lo, hi = PR.wilson_interval(sum(v), len(v))
        table.append({"peak_Te": T, "d": d, "switched": int(sum(v)), "n": len(v), "P": sum(v) / len(v),
                      "wilson95": [lo, hi]})
    return {"instances": len(sysd["instances"]), "atoms_per_instance": g.n_total // len(sysd["instances"]),
            "steps": steps, "seconds": secs, "spin_steps_per_s": g.n_total * steps / secs, "engine": g.engine,
            "table": table}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--peaks", type=float, nargs="+", default=[800.0, 1100.0, 1400.0, 2000.0])
    ap.add_argument("--ds", type=int, nargs="+", default=[2, 4, 6, 8])
    ap.add_argument("--reps", type=int, default=8)
    ap.add_argument("--n", type=int, default=13)
    ap.add_argument("--sweep", default="symmetric", choices=["symmetric", "merged"])
    a = ap.parse_args()
    res = run(a.peaks, a.ds, a.reps, n=a.n, sweep=a.sweep)
    for row in res["table"]:
        print("T_e0 %6.0f K  d %d  P = %d/%d = %.2f  Wilson 95%% [%.2f, %.2f]" % (
            row["peak_Te"], row["d"], row["switched"], row["n"], row["P"], *row["wilson95"]))
    print(json.dumps({k: v for k, v in res.items() if k != "table"}))


if __name__ == "__main__":
    main()
