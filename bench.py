#!/usr/bin/env python
"""Throughput benchmark of the stochastic spin advance (one JSON line).

Workload (default): GdFeCo on a simple-cubic 128^3 lattice (2,097,152 spins)
x 4 realisations, random 25 % Gd, constant nearest-neighbour exchange, a
16^3 TTM grid with a Gaussian laser spot (sigma 40 A) calibrated to a 2000 K
peak, FP32 spins with FP64 TTM, sigma-table and reductions, dt = 0.1 fs.
One benchmark step = `--chunk` time steps of every spin of every realisation,
with the observables (per-sublattice magnetisation, energies, spin
temperature, mean T_e and T_l, FP64) sampled every `--sample-every` steps
(default: once per chunk) inside the timed region.

Metric: spin-steps/s (one spin advanced by one full dt) over all GPUs, with
the fraction of the HBM roofline of the dominant kernel.  The reference arm
(`--impl reference`) times the FP64 CPU oracle on a bounded sample of the
same workload (one realisation, one dt per benchmark step).
"""
import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_SPIN_STEP = {32: 25.0, 64: 49.0}   # read s + write s + species byte


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _workload(name):
    from paper_2608_18541_b300 import workloads as W
    if name == "gdfeco_128x4":
        sysd, ttm = W.config_gdfeco_large(128, 4)
        return sysd, ttm, "GdFeCo sc 128^3 x 4 realisations, 16^3 TTM grid, Gaussian spot 40 A, peak 2000 K"
    if name == "gdfeco_128x1":
        sysd, ttm = W.config_gdfeco_large(128, 1)
        return sysd, ttm, "GdFeCo sc 128^3 x 1 realisation, 16^3 TTM grid, Gaussian spot 40 A, peak 2000 K"
    if name == "gdfeco_256x1":
        sysd, ttm = W.config_gdfeco_large(256, 1)
        return sysd, ttm, "GdFeCo sc 256^3 x 1 realisation, 16^3 TTM grid, Gaussian spot 40 A, peak 2000 K"
    if name == "gdfeco_32":
        sysd, ttm = W.config_gdfeco_32()
        return sysd, ttm, "GdFeCo sc 32^3, one-cell 2TM, 50 fs pulse to 1500 K"
    raise SystemExit("unknown workload " + name)


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to TTS_CLOCK_LOG when set (kept), else to a temporary file
        self.path = os.environ.get("TTS_CLOCK_LOG") or os.path.join(
            tempfile.gettempdir(), "tts_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6400.0, "fallback"


def _record(kernel, precision):
    """The committed ncu record of the dominant kernel (profiles/traffic.json),
    or None when it does not match the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    e = t.get("%s_fp%d" % (kernel, precision))
    if not e:
        return None
    import hashlib
    h = hashlib.sha256()
    try:
        for name in e["sources"]:
            with open(os.path.join(ROOT, "paper_2608_18541_b300", "csrc", name), "rb") as f:
                h.update(f.read())
    except (OSError, KeyError):
        return None
    return e if h.hexdigest()[:16] == e.get("sources_sha") else None


def _traffic(kernel, precision):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    record, or None when it does not match the current kernel sources."""
    e = _record(kernel, precision)
    return e["bytes_per_launch"] if e else None


def _issue(kernel, precision, avg_launch_ms, clocks):
    """Instruction-issue roofline of the dominant kernel: its warp instructions
    per launch (committed ncu record) over the live launch time, against
    4 schedulers x SMs x the SM clock measured during the timed region."""
    e = _record(kernel, precision)
    if not e or not e.get("warp_inst_per_launch") or not avg_launch_ms:
        return None
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = clocks["sm_mhz"] if clocks and clocks.get("sm_mhz") else None
    if not mhz:
        return None
    achieved = e["warp_inst_per_launch"] / (avg_launch_ms / 1e3)
    peak = 4.0 * sms * mhz * 1e6
    return {"achieved": achieved, "peak": peak, "unit": "warp instructions/s", "frac": achieved / peak,
            "warp_inst_per_launch": e["warp_inst_per_launch"], "sm_mhz": mhz, "sms": sms}


def ensemble_leg(P, W, stream, steps=200, sample=64):
    """Batched FP32 ensemble (1024 GdFeCo instances of uneven size in one
    persistent launch per call) against the plain FP64 path that advances one
    instance per launch sequence, on the same GPU."""
    import torch

    sysd, ttm = W.config_ensemble()
    g = P.System(sysd, ttm, precision=32, engine="auto", stream=stream.cuda_stream)
    g.step(5)
    g.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    batched = g.n_total * steps / (e0.elapsed_time(e1) / 1e3)
    engine = g.engine
    del g
    # FP64, one instance per system, instances advanced one after another
    picks = list(range(0, len(sysd["instances"]), len(sysd["instances"]) // sample))[:sample]
    spins, ms = 0, 0.0
    for k in picks:
        one = dict(sysd, instances=[sysd["instances"][k]])
        g1 = P.System(one, ttm, precision=64, engine="general", stream=stream.cuda_stream, instance_base=k)
        g1.step(2)
        g1.sync()
        e0.record(stream)
        g1.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        spins += g1.n_total
        del g1
    fp64 = spins * steps / (ms / 1e3)
    return {"workload": "GdFeCo ensemble, 8 peak T_e x 8 FWHM x 16 realisations = 1024 instances, "
                        "L ~ U{12..24}, x ~ U[0.2, 0.3], one-cell 2TM each",
            "batched_fp32": batched, "batched_engine": engine,
            "fp64_one_instance_per_launch": fp64, "fp64_sample": "%d instances, %d steps each" % (len(picks), steps),
            "ratio": batched / fp64, "unit": "spin-steps/s"}


def merged_leg(P, sysd, ttm, args, stream, spins):
    """The same workload with the merged (leapfrog) sweep: 2 colour passes a
    step instead of 3, the sweep closed at every sample (once per chunk).  A
    different integrator of the same order, reported beside the headline."""
    import torch
    g = P.System(dict(sysd, sweep="merged"), ttm, precision=args.precision, engine=args.engine,
                 stream=stream.cuda_stream)
    for _ in range(args.warmup):
        g.step(args.chunk)
    g.sync()
    steps = max(1, min(args.steps, 10))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g.step(args.chunk)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    del g
    return {"value": spins * steps * args.chunk / (ms / 1e3), "unit": "spin-steps/s",
            "ms_per_step": ms / steps, "steps": steps, "passes_per_dt": 2,
            "note": "sweep closed at every sampling step (once per chunk) and at the end of every call"}


def _launches_per_dt(g, chunk):
    a = g.info().kernel_launches
    g.profile_enable(True)            # direct launches, so that every kernel is counted
    g.step(chunk)
    g.sync()
    ms, steps, ss = g.profile_read()
    g.profile_enable(False)
    return (g.info().kernel_launches - a) / chunk, ms, steps, ss


def fused_leg(P, g, args, stream, spins, peak, peak_kind):
    """The same system with the fused symmetric sweep (checker_sweep_kernel:
    the three colour passes of a step in one launch).  The FP32 checker engine
    offers it last among its launch configurations, one per fusion depth (z
    segments per instance), the cost model's choice last of all.  Every fused
    configuration is timed; the fastest is reported with its whole-step rate,
    the roofline of its launch, and the DRAM traffic of one launch when the ncu
    record matches the sources.  Bitwise the same spins as the headline's
    separate passes; reported beside it."""
    import torch
    cur, n = g.set_config(-1)
    if g.engine != "checker" or args.precision != 32 or n < 2:
        return None
    # the fused configurations launch one spin kernel a step instead of three
    fused = []
    for k in range(n - 1, -1, -1):
        g.set_config(k)
        per, kms, ksteps, kss = _launches_per_dt(g, args.chunk)
        if fused and per != fused[0][1]:
            break
        fused.append((k, per, kms, ksteps, kss))
    steps = max(1, min(args.steps, 5))
    rates = {}
    best = None
    for k, per_step, kms, ksteps, kss in fused:
        g.set_config(k)
        g.step(args.chunk)
        g.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            g.step(args.chunk)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        rates[str(k)] = spins * steps * args.chunk / (ms / 1e3)
        if best is None or ms < best[0]:
            best = (ms, k, per_step, kms, ksteps, kss)
    g.set_config(cur)
    ms, k, per_step, kms, ksteps, kss = best
    bpu = BYTES_PER_SPIN_STEP[args.precision]
    step_ms = ms / (steps * args.chunk)             # the timed region, per dt
    achieved = bpu * spins / (step_ms / 1e3) / 1e9
    return {"value": spins * steps * args.chunk / (ms / 1e3), "unit": "spin-steps/s", "ms_per_step": ms / steps,
            "steps": steps, "kernels_per_dt": per_step, "config": k, "configs_timed": rates,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": _traffic("step_checker_sweep", args.precision),
                         "kernel": "checker_sweep_kernel", "bytes_per_unit": bpu, "units_per_launch": spins,
                         "avg_launch_ms": step_ms, "launch": "one time step, timed region",
                         "kernel_profiled_ms_per_dt": kms / max(ksteps, 1)}}


# ---------------------------------------------------------------------------
# The other workloads of the benchmark suite, each timed on the GPU and
# compared with the FP64 oracle over a short window from the same initial
# state: bcc Fe 10^3 (FP64), GdFeCo 32^3 with a one-cell 2TM (FP64 and FP32)
# and the moving bcc Fe 40^3 lattice (FP32 spins, FP64 TTM).
# ---------------------------------------------------------------------------
def _suite(W):
    """(name, system, ttm, lattice, precisions, timed steps, parity steps, unit)
    of each suite workload; the moving lattice's steps are lattice steps of 10
    spin sub-steps, and its source power is given (no calibration run)."""
    c1 = W.config_bcc_fe_2000()
    c2, t2 = W.config_gdfeco_32()
    c4, t4, l4 = W.config_moving_fe(40)
    t4 = dict(t4, source="power", P0=2e21)
    return [
        ("bcc Fe 10^3 cells (2000 spins), Bethe-Slater NN+NNN, 300 K, no TTM", c1, None, None, (64,), 1000, 200, 1),
        ("GdFeCo sc 32^3 (32768 spins), one-cell 2TM, 50 fs pulse to 1500 K", c2, t2, None, (64, 32), 2000, 200, 1),
        ("moving bcc Fe 40^3 cells (128000 atoms), Morse + magneto-mechanical force, 10x10x40 TTM, "
         "100 fs pulse, source power 2e21 W/m^3", c4, t4, l4, (32,), 10, 2, 10),
    ]


def _oracle_suite(q):
    """Oracle spins after each suite workload's parity window (spawned process)."""
    import oracle as O
    from paper_2608_18541_b300 import workloads as W
    out = []
    for name, sysd, ttm, lat, precs, steps, psteps, sub in _suite(W):
        t0 = time.perf_counter()
        o = O.Oracle(sysd, ttm, lattice=lat)
        if lat is not None:
            o.lattice_step(psteps)
        else:
            o.step(psteps)
        out.append((o.spins(), time.perf_counter() - t0))
    q.put(out)


class OracleSuite:
    def __init__(self):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.q = ctx.Queue()
        self.proc = ctx.Process(target=_oracle_suite, args=(self.q,))
        self.proc.start()

    def result(self, timeout=3600):
        r = self.q.get(timeout=timeout)
        self.proc.join()
        return r


def suite_leg(P, W, stream, oracle):
    """Throughput and FP64-oracle parity of the suite workloads on the GPU."""
    import numpy as np
    import torch
    gpu = []
    for name, sysd, ttm, lat, precs, steps, psteps, sub in _suite(W):
        for prec in precs:
            g = P.System(sysd, ttm, precision=prec, stream=stream.cuda_stream, lattice=lat)
            g.step(psteps)
            got = g.get_spins(0)
            g.step(max(1, steps // 10))
            g.sync()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            gpu.append((name, prec, g.engine, g.n_total, steps, sub, ms, psteps, got))
            del g
    want = oracle.result()
    idx = {n: k for k, (n, *_rest) in enumerate(_suite(W))}
    out = []
    for name, prec, engine, n, steps, sub, ms, psteps, got in gpu:
        ref, osec = want[idx[name]]
        tol = 1e-10 if prec == 64 else 2e-5
        err = float(np.abs(got - ref).max())
        out.append({"workload": name, "precision": "f%d" % prec, "engine": engine, "spins": n,
                    "value": n * steps * sub / (ms / 1e3), "unit": "spin-steps/s",
                    "timed": "%d %s" % (steps, "lattice steps (x%d spin sub-steps)" % sub if sub > 1 else "steps"),
                    "parity": {"max_abs_ds": err, "tolerance": tol, "pass": err <= tol,
                               "steps": psteps if sub == 1 else "%d lattice steps" % psteps,
                               "against": "FP64 CPU oracle, same seeds, per spin component"}})
    return out


# ---------------------------------------------------------------------------
# The FP64 CPU oracle on the host cores, the paper's task-level strategy: one
# single-threaded process per realisation, all running at once.  Everything
# here runs in spawned interpreters (no CUDA state is ever forked).
# ---------------------------------------------------------------------------
def _pool_size(want=None):
    n = os.cpu_count() or 1
    p = max(1, n - 2) if want is None else max(1, want)
    try:
        import psutil
        p = min(p, max(1, int(psutil.virtual_memory().available // (600 << 20))))
    except (ImportError, OSError):
        pass
    return min(p, 64)


def _oracle_worker(sysd, ttm, instance, warm, steps, barrier, q):
    import oracle as O
    o = O.Oracle(sysd, ttm, instance=instance, index=0)
    o.step(warm)
    barrier.wait(timeout=900)
    t0 = time.perf_counter()
    o.step(steps)
    q.put((instance, o.n, steps, time.perf_counter() - t0))


def _oracle_campaign(sysd, ttm, nproc, warm, steps, parity_steps, q):
    """Calibrate the source power once (oracle, realisation 0), run `nproc`
    concurrent single-threaded oracles (realisations 0..nproc-1, the source
    power as calibrated) for `warm` + `steps` time steps, and, when
    parity_steps > 0, advance one more realisation-0 oracle from the initial
    state by parity_steps steps and report its spins."""
    import multiprocessing as mp
    import numpy as np
    import oracle as O
    one = dict(sysd)
    if one.get("instances"):
        one["instances"] = one["instances"][:1]
    t0 = time.perf_counter()
    cal = O.Oracle(one, ttm, instance=0, index=0)
    calib_s = time.perf_counter() - t0
    tp = dict(ttm, source="power", P0=cal.P0) if ttm and ttm.get("source") == "peak" else ttm
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(nproc)
    rq = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(one, tp, k, warm, steps, barrier, rq)) for k in range(nproc)]
    for pr in procs:
        pr.start()
    spins = None
    if parity_steps > 0:
        cal.step(parity_steps)
        spins = cal.spins()
    res = [rq.get(timeout=1800) for _ in procs]
    for pr in procs:
        pr.join()
    n_each = res[0][1]
    wall = max(r[3] for r in res)
    q.put({"nproc": nproc, "n_each": n_each, "steps": steps, "warm": warm, "wall_s": wall,
           "aggregate": sum(r[1] * r[2] for r in res) / wall,
           "per_core": float(np.mean([r[1] * r[2] / r[3] for r in res])),
           "calibration_s": calib_s, "P0": cal.P0})
    q.put(spins)


class OracleCampaign:
    """The CPU side started in the background (a spawned process), read later."""

    def __init__(self, sysd, ttm, nproc, warm, steps, parity_steps=0):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.q = ctx.Queue()
        self.nproc = nproc
        self.proc = ctx.Process(target=_oracle_campaign,
                                args=(sysd, ttm, nproc, warm, steps, parity_steps, self.q))
        self.proc.start()

    def result(self, timeout=3600):
        stats = self.q.get(timeout=timeout)
        spins = self.q.get(timeout=timeout)
        self.proc.join()
        return stats, spins


def single_leg(P, W, n, args, stream, peak, peak_kind):
    """One realisation of the workload's model at n^3 (the single-instance
    roofline case; 256^3 holds 268 MB of state, twice L2): spin-steps/s of the
    whole step and the roofline of the colour passes."""
    import torch
    sysd, ttm = W.config_gdfeco_large(n, 1)
    sample_every = args.chunk if args.sample_every < 0 else args.sample_every
    sysd = dict(sysd, sample_every=sample_every)
    g = P.System(sysd, ttm, precision=args.precision, engine=args.engine, stream=stream.cuda_stream)
    g.step(args.chunk)
    g.sync()
    steps = max(1, min(args.steps, 5))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g.step(args.chunk)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    g.profile_enable(True)
    g.step(2 * args.chunk)
    g.sync()
    kms, ksteps, kss = g.profile_read()
    g.profile_enable(False)
    bpu = BYTES_PER_SPIN_STEP[args.precision]
    step_ms = ms / (steps * args.chunk)             # the timed region, per dt
    achieved = bpu * g.n_total / (step_ms / 1e3) / 1e9
    out = {"workload": "GdFeCo sc %d^3 x 1 realisation, 16^3 TTM grid, Gaussian spot 40 A, peak 2000 K" % n,
           "spins": g.n_total, "value": g.n_total * steps * args.chunk / (ms / 1e3), "unit": "spin-steps/s",
           "ms_per_step": ms / steps, "steps": steps, "dt_per_step": args.chunk, "engine": g.engine,
           "l2": "state %.0f MB vs L2 126 MB" % (g.n_total * 16 / 1e6),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "peak_kind": peak_kind,
                        "traffic": _traffic("step_%s_%dx1" % (g.engine, n), args.precision),
                        "kernel": "step_" + g.engine, "bytes_per_unit": bpu, "units_per_launch": g.n_total,
                        "avg_launch_ms": step_ms, "launch": "one time step, timed region",
                        "passes_profiled_ms_per_dt": kms / max(ksteps, 1)}}
    del g
    return out


def _cpu_sample_text(st):
    return ("%d concurrent single-threaded FP64 oracle processes (the paper's one process per "
            "realisation), realisation k = 0..%d of the workload's model (%d spins each), %d timed "
            "step(s) of dt after %d warm-up step(s) each; value = all spin-steps / the slowest "
            "process's time; source power calibrated once by the oracle (%.0f s, not timed)" % (
                st["nproc"], st["nproc"] - 1, st["n_each"], st["steps"], st["warm"], st["calibration_s"]))


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    sysd, ttm, desc = _workload(args.workload)
    sample_every = args.chunk if args.sample_every < 0 else args.sample_every
    sysd = dict(sysd, sample_every=sample_every)
    camp = OracleCampaign(sysd, ttm, _pool_size(args.cpu_procs), args.warmup, args.steps)
    st, _ = camp.result()
    v = st["aggregate"]
    cpu = {"value": v, "unit": "spin-steps/s", "cores": st["nproc"], "nproc": os.cpu_count(), "kind": "oracle",
           "per_core": st["per_core"], "aggregate": v, "sample": _cpu_sample_text(st)}
    line = {
        "impl": "reference", "metric": "spin-steps/s", "value": v, "unit": "spin-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * st["wall_s"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "sample_every": sample_every,
                                              "sample": "one dt per step on every process"},
        "cpu_baseline": cpu,
        "e2e": {"value": v, "unit": "spin-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--chunk", type=int, default=100, help="time steps per benchmark step")
    ap.add_argument("--sample-every", type=int, default=-1,
                    help="observable sampling interval in time steps (default: once per chunk; 0: off)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gdfeco_128x4")
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--engine", default="auto")
    ap.add_argument("--cpu-steps", type=int, default=3, help="timed oracle steps per CPU process")
    ap.add_argument("--cpu-procs", type=int, default=None, help="oracle processes (default: host cores - 2)")
    ap.add_argument("--parity-steps", type=int, default=100,
                    help="steps of realisation 0 compared with the FP64 oracle (0: none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-single", action="store_true", help="skip the single-instance roofline legs")
    ap.add_argument("--no-fused", action="store_true", help="skip the fused-sweep leg")
    ap.add_argument("--config", default="-1",
                    help="launch configuration of the timed system (tts_set_config index; -1: the default; "
                         "'last': the last one offered, for the FP32 checker the fused sweep at the cost "
                         "model's fusion depth)")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-suite", action="store_true", help="skip the other workloads of the suite")
    ap.add_argument("--no-merged", action="store_true")
    args = ap.parse_args()

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import numpy as np

    import paper_2608_18541_b300 as P
    from paper_2608_18541_b300 import build as B

    if not os.path.exists(P.LIB_PATH):
        B.build()
    sysd, ttm, desc = _workload(args.workload)
    # the per-sample reductions (magnetisation per sublattice, energies, spin
    # temperature, mean T_e and T_l) are part of the timed path
    sample_every = args.chunk if args.sample_every < 0 else args.sample_every
    sysd = dict(sysd, sample_every=sample_every)
    n_inst_local = len(sysd.get("instances") or [0])
    stream = torch.cuda.current_stream()
    g = P.System(sysd, ttm, precision=args.precision, engine=args.engine, stream=stream.cuda_stream,
                 instance_base=rank * n_inst_local)
    spins = g.n_total
    if args.config == "last":
        g.set_config(g.set_config(-1)[1] - 1)
    elif int(args.config) >= 0:
        g.set_config(int(args.config))
    initial = g.get_state()
    for _ in range(args.warmup):
        g.step(args.chunk)
    g.sync()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    sampler = ClockSampler(local) if local == 0 else None
    launches0 = g.info().kernel_launches
    barrier()
    if sampler:
        sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        g.step(args.chunk)
    ev1.record(stream)
    barrier()
    clocks = sampler.stop() if sampler else None
    ms = ev0.elapsed_time(ev1)
    launches = g.info().kernel_launches - launches0
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    tot = torch.tensor([float(spins)], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    total_spins = float(tot.item())
    total_dt = args.steps * args.chunk
    value = total_spins * total_dt / (ms_max / 1e3)

    # device time of the colour-pass launches alone (events around them), in a
    # separate profiled run after the timed one (reported for information: the
    # roofline below is taken over the timed region itself)
    g.profile_enable(True)
    for _ in range(min(args.steps, 5)):
        g.step(args.chunk)
    g.sync()
    kern_ms, kern_steps, kern_spin_steps = g.profile_read()
    g.profile_enable(False)

    # end to end through the public API with host buffers: every benchmark
    # step uploads the state from page-locked host memory, advances it and
    # reads the spins and one observable row back, the state flowing through
    # the host from step to step
    rdt = torch.float32 if args.precision == 32 else torch.float64
    bufs = [torch.empty((spins, 3), dtype=rdt, pin_memory=True).numpy() for _ in range(2)]
    g.read_spins_async(bufs[0])
    g.sync()
    barrier()
    t0 = time.perf_counter()
    cur = 0
    for _ in range(args.steps):
        g.write_spins_async(bufs[cur])
        g.step(args.chunk)
        g.read_spins_async(bufs[1 - cur])
        obs = g.observe_now(0)           # synchronises: the read-back is complete
        cur = 1 - cur
    barrier()
    e2e_s = time.perf_counter() - t0
    te = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_s = float(te.item())
    e2e = {"value": total_spins * total_dt / e2e_s, "unit": "spin-steps/s",
           "h2d_bytes_per_step": int(bufs[0].nbytes),
           "d2h_bytes_per_step": int(bufs[0].nbytes + obs.nbytes),
           "note": "per step: state upload from page-locked memory, the step, spins and observables read back"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # the CPU side (oracle on the host cores, and the oracle trajectory the
    # parity check compares with) runs in the background from here on
    camp = None
    if world == 1 and not args.no_cpu_baseline:
        camp = OracleCampaign(sysd, ttm, _pool_size(args.cpu_procs), 1, args.cpu_steps, args.parity_steps)
    osuite = OracleSuite() if world == 1 and not args.no_suite else None

    peak, peak_kind = _peaks()
    bpu = BYTES_PER_SPIN_STEP[args.precision]
    kernel_name = "step_" + g.engine
    # One launch = one time step of the path (the colour passes of every
    # instance, with the TTM beside them and the sampled observables), its
    # duration from the CUDA events of the timed region: ms per dt.
    step_ms = ms_max / total_dt
    achieved = bpu * spins / (step_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind,
                "traffic": _traffic(kernel_name, args.precision), "kernel": kernel_name,
                "bytes_per_unit": bpu, "units_per_launch": spins, "avg_launch_ms": step_ms,
                "launch": "one time step (all colour passes of every instance), timed region",
                "passes_profiled_ms_per_dt": kern_ms / max(kern_steps, 1) if kern_ms > 0 else None}
    # the kernel is bound by instruction issue: the same launch against that ceiling
    roofline["issue"] = _issue(kernel_name, args.precision, roofline["avg_launch_ms"], clocks)
    engine = g.engine
    from paper_2608_18541_b300 import workloads as W
    merged = None
    if world == 1 and not args.no_merged:
        merged = merged_leg(P, sysd, ttm, args, stream, spins)
    ens = None
    if world == 1 and not args.no_ensemble:
        ens = ensemble_leg(P, W, stream)
    fused = None
    if world == 1 and not args.no_fused:
        fused = fused_leg(P, g, args, stream, spins, peak, peak_kind)
    suite = suite_leg(P, W, stream, osuite) if osuite is not None else None
    single = None
    if world == 1 and not args.no_single and args.workload == "gdfeco_128x4":
        single = [single_leg(P, W, n, args, stream, peak, peak_kind) for n in (128, 256)]
    cpu = parity = None
    if camp is not None:
        # realisation 0 advanced parity_steps from the initial state on the GPU
        if args.parity_steps > 0:
            g.set_state(initial)
            g.step(args.parity_steps)
            got = g.get_spins(0)
        st, want = camp.result()
        cpu = {"value": st["aggregate"], "unit": "spin-steps/s", "cores": st["nproc"], "nproc": os.cpu_count(),
               "kind": "oracle", "per_core": st["per_core"], "aggregate": st["aggregate"],
               "sample": _cpu_sample_text(st)}
        if args.parity_steps > 0:
            tol = 2e-5 if args.precision == 32 else 1e-10
            err = float(np.abs(got - want).max())
            parity = {"max_abs_ds": err, "tolerance": tol, "pass": err <= tol, "steps": args.parity_steps,
                      "realisation": 0, "spins": int(want.shape[0]),
                      "against": "FP64 CPU oracle, same seeds, per spin component"}
    line = {
        "metric": "spin-steps/s", "value": value, "unit": "spin-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
        "config": {"workload": desc, "spins_per_gpu": spins, "dt_per_step": args.chunk,
                   "sample_every": sample_every,
                   "engine": engine, "l2": "state and tables exceed L2 (126 MB) per step" if spins * 16 > 126e6
                   else "working set may fit L2", "parallelism": "instances sharded, dp%d" % world},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clocks, "parity": parity, "single_instance": single, "fused_sweep": fused, "ensemble": ens,
        "merged_sweep": merged, "suite": suite,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
