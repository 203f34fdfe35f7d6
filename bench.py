#!/usr/bin/env python3
"""Throughput of the noise -> Zel'dovich path (grid cells per second) on GB300.

One step = one pass of the whole path over one grid: Philox white noise,
forward r2c 3-D transform, Eq. 1 filter, then for each component j the Eq. 2
filter, the c2r transform and the Eq. 3 epilogue writing positions and
velocities (Ginnungagap, arXiv:2511.10353, Secs. 2.1-2.2).

Default workload: 512^3 cells, L = 500 Mpc/h, BBKS (Om=.3, h=.7, ns=.96,
s8=.8), z = 100, FP32, outputs pos + vel (3 + 3 grids). The working set
(>= 4.3 GB) is far larger than the 129 MB L2, so no flush is needed. The
default run also times the 1536^3 precision workload (2000 Mpc/h,
Eisenstein-Hu no-wiggle, z = 100) with its FP64 path and FP32 error under
the key "zeldovich_1536_fp32" (--no-1536 skips it), and the oracle on the
whole 512^3 workload as the CPU baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

Prints one JSON line (rank 0). Under torchrun each rank runs an independent
replica (the path has no exchange step on one GPU): value = cells of all
ranks / max-over-ranks time, scaling "weak".
"""
import argparse
import hashlib
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

METRIC = "grid cells/sec noise->Zel'dovich (FP32 vs FP64 plain), % HBM roofline, err vs FP64"
FALLBACK_HBM_GBS = 6800.0

# dram bytes (read + write) per launch of the dominant kernel from one ncu
# capture, scaled to the bench workload, with the hash of the kernel sources it
# was taken on; reported as null when the sources have changed since.
NCU_TRAFFIC = {
    # profiles/z_inverse_512_fp32_ncu.md: 536,953,344 B read + 1,015,245,000 B written
    ("z_inverse_epilogue", "zeldovich_512_fp32"): (1552198344.0, "9c66d602be30deff"),
    # the same capture scaled to a 1536^3 launch by the cells processed (x 27):
    # a multi-counter capture at full size is beyond the pool's capture limits
    ("z_inverse_epilogue", "zeldovich_1536_fp32"): (41909355288.0, "9c66d602be30deff"),
}


def kernel_source_hash():
    """Hash of the kernel headers' code (// comments and blank lines left out,
    so that a comment edit keeps the recorded ncu traffic valid)."""
    h = hashlib.sha256()
    for f in ("gg_device.cuh", "gg_kernels.cuh", "gg_ct.cuh", "gg_ct_kernels.cuh"):
        with open(os.path.join(ROOT, "paper_2511_10353_gb300", "csrc", f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="zeldovich_512_fp32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-1536", action="store_true",
                    help="skip the 1536^3 leg of the default run")
    ap.add_argument("--variants", default=None,
                    help="comma list of 6 tile variants instead of autotuning (profiling runs)")
    ap.add_argument("--layout", choices=["auto", "plain", "chunked"], default="auto",
                    help="spectrum layout between the y passes (auto: the autotuner's choice; "
                         "with --variants, plain unless given)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def config_of(w, outputs="pos+vel"):
    return {"workload": "zeldovich_%d_%s" % (w["n"], w["prec"].replace("f", "fp")),
            "n": w["n"], "box_mpc_h": w["box"], "transfer": w["cosmo"]["tf"],
            "omega_m": w["cosmo"]["omega_m"], "z_init": w["z_init"], "outputs": outputs,
            "cells_per_step": w["n"] ** 3,
            "l2": "working set > L2 (129 MB), no flush", "parallelism": "replicas"}


# ------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------ CPU baseline
def oracle_sample(w, n_s):
    """The oracle on an n_s^3 grid with the workload's cell size: (seconds, cells)."""
    from oracle import fields
    from oracle.cosmology import Cosmology
    c = w["cosmo"]
    cosmo = Cosmology(c["omega_m"], c["h"], c["n_s"], c["sigma_8"], tf=c["tf"],
                      omega_b=c.get("omega_b", 0.049), t_cmb=c.get("t_cmb", 2.7255))
    cosmo.amplitude()
    box = w["box"] * n_s / w["n"]
    t0 = time.perf_counter()
    fields.zeldovich(n_s, box, cosmo, w["z_init"], seed=w["seed"])
    return time.perf_counter() - t0, n_s ** 3


def cpu_baseline(w, n_s=256):
    from oracle.fields import WORKERS
    secs, cells = oracle_sample(w, n_s)
    what = ("one step of the workload itself (%d^3, box %.1f Mpc/h, seed %d)" % (n_s, w["box"], w["seed"])
            if n_s == w["n"] else
            "one %d^3 realization (box %.1f Mpc/h, same cell size and cosmology)"
            % (n_s, w["box"] * n_s / w["n"]))
    return {"value": cells / secs, "unit": "cells/s", "cores": WORKERS, "kind": "oracle",
            "sample": what + ", all three components' psi, pos and vel, FP64 numpy/scipy; "
                      "noise single-threaded, FFTs on %d scipy workers; %.1f s" % (WORKERS, secs)}


def run_reference(args, w):
    rank, _, world = dist_env()
    if rank != 0:
        return
    per_step_budget = 150.0 / max(1, args.steps + args.warmup)
    n_s = 128 if per_step_budget >= 1.5 else (64 if per_step_budget >= 0.15 else 32)
    for _ in range(args.warmup):
        oracle_sample(w, n_s)
    total, cells = 0.0, 0
    for _ in range(args.steps):
        s, c = oracle_sample(w, n_s)
        total += s
        cells += c
    value = cells / total
    from oracle.fields import WORKERS
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w),
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": WORKERS, "kind": "oracle",
                             "sample": "each step one %d^3 realization with the workload's cell "
                                       "size and cosmology (FP64 numpy/scipy oracle)" % n_s},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- batched form
def run_batched(args):
    """48 realizations (N cycling 128/192/256/384, L = N Mpc/h, seeds 1..48,
    FP32, pos + vel) in one CUDA graph, timed in both batched schedules: one
    launch per pass and size group, and one persistent launch over every pass
    and realization. The line's value is the faster; both are reported."""
    import torch
    import paper_2511_10353_gb300 as gg
    from paper_2511_10353_gb300 import build
    from paper_2511_10353_gb300.workloads import batched_realizations
    torch.cuda.set_device(0)
    build.build(verbose=False)
    specs = batched_realizations()
    b = gg.Batch(specs)
    t = time.perf_counter()
    b.autotune(2)
    t_tune = time.perf_counter() - t
    out = b.empty_outputs()
    seeds = [w["seed"] for w in specs]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(persistent):
        b.set_persistent(persistent)
        t = time.perf_counter()
        b.run(seeds, out)  # the first run captures the graph
        b.sync()
        capture = time.perf_counter() - t
        for _ in range(max(3, args.warmup)):
            b.run(seeds, out)
        b.sync()
        sampler = ClockSampler(0)
        sampler.start()
        e0.record(b.stream)
        for i in range(args.steps):
            b.run([s + i for s in seeds], out)
        e1.record(b.stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1) / args.steps
        return {"ms_per_step": ms, "value": b.cells / (ms * 1e-3), "unit": "cells/s",
                "gpu_launches_per_step": b.launches(), "graph_capture_s": round(capture, 3),
                "clocks": clocks}

    per_pass = timed(False)
    per_pass["schedule"] = "one launch per pass and size group, groups on forked streams"
    persistent = timed(True)
    persistent["schedule"] = ("one persistent launch: work items (pass, group, run of tiles) "
                              "in order from a device counter, per-realization pass counters")
    best, other = (persistent, per_pass) if persistent["ms_per_step"] <= per_pass["ms_per_step"] \
        else (per_pass, persistent)
    ms, value = best["ms_per_step"], best["value"]
    peak, src = peak_hbm()
    gbs = 80.0 * b.cells / (ms * 1e-3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched_48", "realizations": len(specs),
                       "sizes": [128, 192, 256, 384], "box": "N Mpc/h", "z_init": 50.0,
                       "outputs": "pos+vel", "cells_per_step": b.cells, "groups": b.groups,
                       "schedule": best["schedule"], "graph_capture_s": best["graph_capture_s"],
                       "autotune_s": round(t_tune, 3),
                       "l2": "working set > L2 (129 MB), no flush", "parallelism": "replicas"},
            "path": {"algorithmic_bytes_per_cell": 80.0, "GB_s": gbs, "frac_of_peak": gbs / peak,
                     "peak_source": src},
            "gpu_launches": best["gpu_launches_per_step"] * args.steps, "clocks": best["clocks"],
            "other_schedule": other}
    b.close()
    if not args.no_cpu_baseline:  # the oracle on the batch's first two realizations, in turn
        from oracle.fields import WORKERS
        secs = cells = 0
        for w in specs[:2]:
            t_s, c_s = oracle_sample(w, w["n"])
            secs += t_s
            cells += c_s
        line["cpu_baseline"] = {
            "value": cells / secs, "unit": "cells/s", "cores": WORKERS, "kind": "oracle",
            "sample": "realizations 1-2 of the batch (128^3 and 192^3, seeds 1-2), one after "
                      "the other, FP64 numpy/scipy; FFTs on %d scipy workers; %.1f s"
                      % (WORKERS, secs)}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ white-noise refinement
REFINE_METRIC = "child grid cells/sec, white-noise refinement (Appendix A), % HBM roofline"


def refine_cpu_sample(w, n_s):
    """The oracle refinement of an n_s^3 parent: (seconds, child cells)."""
    from oracle import noise, refine
    parent = noise.white_noise(w["seed_parent"], n_s)
    t0 = time.perf_counter()
    child = refine.refine(parent, w["kind"], w["seed_child"])
    return time.perf_counter() - t0, child.size


def run_refine(args):
    """gg_refine_noise on the workload's parent grid, one launch per step."""
    import torch
    import paper_2511_10353_gb300 as gg
    from paper_2511_10353_gb300 import build
    from paper_2511_10353_gb300.workloads import BBKS, REFINE_WORKLOADS
    w = REFINE_WORKLOADS[args.workload]
    rank, _, world = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return
        n_s = 32  # about 0.3 s per step on one core
        for _ in range(args.warmup):
            refine_cpu_sample(w, n_s)
        total, cells = 0.0, 0
        for _ in range(args.steps):
            s, c = refine_cpu_sample(w, n_s)
            total += s
            cells += c
        from oracle.fields import WORKERS
        value = cells / total
        print(json.dumps({
            "impl": "reference", "metric": REFINE_METRIC, "value": value, "unit": "cells/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n_parent": w["n"], "kind": w["kind"]},
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": 1, "kind": "oracle",
                             "sample": "each step one %d^3 parent refined by the numpy oracle"
                                       % n_s},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}), flush=True)
        return
    torch.cuda.set_device(0)
    build.build(verbose=False)
    n = w["n"]
    dtype = torch.float32 if w["prec"] == "f32" else torch.float64
    esz = 4 if w["prec"] == "f32" else 8
    plan = gg.Plan(n, float(n), BBKS, 50.0, w["prec"])
    parent = plan.white_noise(seed=w["seed_parent"])
    plan.sync()
    plan.close()
    dims = gg.refine_dims(n, w["kind"])
    child = torch.empty(dims, dtype=dtype, device="cuda")
    cells = dims[0] * dims[1] * dims[2]
    for i in range(max(3, args.warmup)):
        gg.refine_noise(parent, w["seed_child"] + i, w["kind"], out=child)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        gg.refine_noise(parent, w["seed_child"] + i, w["kind"], out=child)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    value = cells / (ms * 1e-3)
    nbytes = esz * (n ** 3 + cells)  # parent read once, child written once
    peak, src = peak_hbm()
    achieved = nbytes / (ms * 1e-3) / 1e9
    line = {"metric": REFINE_METRIC, "value": value, "unit": "cells/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": w["prec"], "data": "synthetic",
            "config": {"workload": args.workload, "n_parent": n, "child_dims": list(dims),
                       "kind": w["kind"], "cells_per_step": cells,
                       "l2": "working set > L2 (129 MB), no flush"},
            "roofline": {"bound": "hbm", "kernel": "k_refine", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_source": src,
                         "algorithmic_bytes_per_launch": nbytes, "traffic": None},
            "gpu_launches": args.steps, "clocks": clocks, "e2e": None}
    if not args.no_cpu_baseline:
        secs, c = refine_cpu_sample(w, 64)
        line["cpu_baseline"] = {"value": c / secs, "unit": "cells/s", "cores": 1, "kind": "oracle",
                                "sample": "one 64^3 parent refined by the numpy oracle (%.1f s)"
                                          % secs}
    print(json.dumps(line), flush=True)


# ---------------------------------------------- the operations beyond the path
FEATURES_METRIC = "ms and algorithmic GB/s per call of the Sec. 2.1-2.4 operations at 512^3 FP32"


def run_features(args):
    """Times each operation around the main path once per step (CUDA events on
    the current stream): the Sec. 2.4 large-scale filter (256^3) and merge
    (512^3 with 256^3 large scales), gas pairs, degrading 512^3 -> 256^3, the
    power spectrum, coordinate IDs and the Appendix A refinement 256^3 ->
    512^3. Algorithmic bytes (FP32) per call are stated per operation."""
    import torch
    import paper_2511_10353_gb300 as gg
    from paper_2511_10353_gb300 import build
    from paper_2511_10353_gb300.workloads import BBKS
    torch.cuda.set_device(0)
    build.build(verbose=False)
    n, nl, box, z = 512, 256, 500.0, 100.0
    hi = gg.Plan(n, box, BBKS, z, "f32")
    lo = gg.Plan(nl, box, BBKS, z, "f32")
    hi.autotune(2)
    lo.autotune(2)
    r_s = 2 * box / nl
    psi_lo = lo.zeldovich(seed=1, pos=False, vel=False)["psi"]
    large = [lo.empty() for _ in range(3)]
    out = hi.zeldovich(seed=2)
    gas = [hi.empty() for _ in range(3)]
    ids = torch.empty((n, n, n), dtype=torch.int64, device="cuda")
    coarse = lo.empty()
    delta = hi.gaussian_field(seed=3)
    parent = lo.white_noise(seed=4)
    child = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    c, cl = n ** 3, nl ** 3
    ops = {
        "large_scales_256": (lambda: [lo.large_scales(psi_lo[j], r_s, out=large[j]) for j in range(3)],
                             3 * 56.0 * cl, "3 components, 56 B/cell: 7 passes"),
        "zeldovich_merge_512": (lambda: hi.zeldovich_merge(large, r_s, seed=2, out=out),
                                80.0 * c + 3 * 4.0 * cl, "80 B/cell + the 256^3 large scales"),
        "zeldovich_gas_512": (lambda: hi.zeldovich_gas(0.163, seed=2, out={"psi": [None] * 3,
                              "pos": out["pos"], "pos_gas": gas, "vel": out["vel"]}),
                              92.0 * c, "80 B/cell + 3 gas position grids"),
        "zeldovich_plain_512": (lambda: hi.zeldovich(seed=2, out=out), 80.0 * c, "the main path"),
        "degrade_512_to_256": (lambda: lo.degrade(delta, out=coarse), 4.0 * cl + 56.0 * cl,
                               "gather + 56 B/coarse cell"),
        "power_spectrum_512": (lambda: hi.power_spectrum(delta), 28.0 * c, "3 forward passes + bins"),
        "particle_ids_512": (lambda: hi.particle_ids(n, 0, out=ids), 8.0 * c, "int64 write"),
        "refine_256_to_512": (lambda: gg.refine_noise(parent, 5, "2", out=child), 4.0 * (cl + c),
                              "parent read + child write"),
    }
    peak, src = peak_hbm()
    res = {}
    stream = torch.cuda.current_stream()
    steps = max(3, min(args.steps, 20))
    for name, (fn, nbytes, note) in ops.items():
        for _ in range(max(2, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        gbs = nbytes / (ms * 1e-3) / 1e9
        res[name] = {"ms": ms, "GB_s": gbs, "frac_of_peak": gbs / peak, "bytes": nbytes, "bytes_note": note}
    line = {"metric": FEATURES_METRIC, "value": res["zeldovich_merge_512"]["ms"], "unit": "ms",
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "features_512", "n": n, "n_low": nl, "box_mpc_h": box,
                       "peak_GB_s": peak, "peak_source": src},
            "features": res}
    for p in (hi, lo):
        p.close()
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def time_plain(gg, w, steps, warmup, variants_arg, world, barrier, gpu_id, allreduce_max,
               layout="auto"):
    """Plan, autotune, warm-up, then `steps` timed steps of noise -> pos + vel
    (CUDA events on the plan's stream, per-kernel events on the same stream,
    clocks sampled meanwhile). Returns (result dict, plan, variants)."""
    import torch
    n = w["n"]
    cells = n ** 3
    plan = gg.Plan(n, w["box"], w["cosmo"], w["z_init"], w["prec"])
    shape = (n, n, n)
    out = {"psi": [None] * 3,
           "pos": [torch.empty(shape, dtype=plan.dtype, device="cuda") for _ in range(3)],
           "vel": [torch.empty(shape, dtype=plan.dtype, device="cuda") for _ in range(3)]}
    stream = torch.cuda.current_stream()
    t_tune = time.perf_counter()
    if variants_arg:
        plan.set_variants([int(v) for v in variants_arg.split(",")])
        variants = plan.variants()
    else:
        variants = plan.autotune(3)  # tile variants per pass, timed on this plan's buffers
    if layout != "auto":
        plan.set_layout(layout == "chunked")
    t_tune = time.perf_counter() - t_tune
    for i in range(max(3, warmup)):
        plan.zeldovich(seed=1 + i, out=out)
    plan.sync()
    plan.set_profiling(True)
    plan.profile(reset=True)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(steps):
        plan.zeldovich(seed=1 + i, out=out)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    plan.sync()
    prof = plan.profile(reset=True)
    plan.set_profiling(False)
    ms = allreduce_max(t0.elapsed_time(t1))
    value = world * cells * steps / (ms * 1e-3)
    launches = sum(v["launches"] for v in prof.values())
    peak, peak_src = peak_hbm()
    kernels = {}
    for name, v in prof.items():
        per = v["ms"] / v["launches"]
        gbs = v["bytes"] / (per * 1e-3) / 1e9
        kernels[name] = {"ms_per_launch": per, "launches": v["launches"], "GB_s": gbs,
                         "frac_of_peak": gbs / peak,
                         "share": v["ms"] / sum(x["ms"] for x in prof.values())}
    dom = max(prof, key=lambda k: prof[k]["ms"])
    dper = prof[dom]["ms"] / prof[dom]["launches"]
    achieved = prof[dom]["bytes"] / (dper * 1e-3) / 1e9
    traffic = None
    rec = NCU_TRAFFIC.get((dom, config_of(w)["workload"]))
    if rec and rec[1] == kernel_source_hash():
        traffic = rec[0]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                "algorithmic_bytes_per_launch": prof[dom]["bytes"], "traffic": traffic}
    if traffic is not None and w["n"] != 512:
        roofline["traffic_source"] = "512^3 ncu capture scaled by the cells processed"
    step_bytes = sum(v["bytes"] * v["launches"] for v in prof.values()) / steps
    path_gbs = step_bytes / (ms / steps * 1e-3) / 1e9
    res = {"value": value, "ms_per_step": ms / steps, "steps": steps,
           "config": dict(config_of(w), tile_variants=variants, autotune_s=round(t_tune, 3),
                          spectrum_layout="chunk-major" if plan.layout() else "plain"),
           "roofline": roofline,
           "path": {"algorithmic_bytes_per_cell": step_bytes / cells, "GB_s": path_gbs,
                    "frac_of_peak": path_gbs / peak},
           "kernels": kernels, "gpu_launches": launches, "clocks": clocks}
    del out
    torch.cuda.empty_cache()
    return res, plan, variants


def fp64_leg(gg, w, plan, value_per_gpu, steps):
    """The FP64 plain path on the same workload: the FP32 psi's relative L2
    error against it, and its own rate. Closes the FP32 plan (its workspaces
    make room for the FP64 grids: 261 GB at 1536^3)."""
    import torch
    n = w["n"]
    cells = n ** 3
    shape = (n, n, n)
    plan64 = gg.Plan(n, w["box"], w["cosmo"], w["z_init"], "f64")
    psi64 = torch.empty(shape, dtype=torch.float64, device="cuda")
    psi32 = torch.empty(shape, dtype=torch.float32, device="cuda")
    errs = []
    for j in range(3):
        sel = lambda t: {"psi": [t if c == j else None for c in range(3)], "pos": [None] * 3,
                         "vel": [None] * 3}
        plan64.zeldovich(seed=1, out=sel(psi64))
        plan.zeldovich(seed=1, out=sel(psi32))
        torch.cuda.synchronize()
        num = den = 0.0
        for x0 in range(0, n, 128):  # slabs bound the FP64 temporaries
            d = psi32[x0:x0 + 128].double() - psi64[x0:x0 + 128]
            num += float((d * d).sum())
            den += float((psi64[x0:x0 + 128] ** 2).sum())
        errs.append(math.sqrt(num / den))
    del psi64, psi32
    err = {"psi_rel_l2": errs, "reference": "GPU FP64 path (within 1e-12 of the FP64 oracle "
           "in tests/test_gpu_fullsize.py, 1e-11 of the oracle's closed form at 1536^3 in "
           "tests/test_gpu_1536.py)"}
    plan.close()
    torch.cuda.empty_cache()
    need = 6 * cells * 8 + (1 << 30)
    out64, why = None, None
    if torch.cuda.mem_get_info()[0] >= need:
        out64 = {"psi": [None] * 3,
                 "pos": [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(3)],
                 "vel": [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(3)]}
        try:  # the plan's own workspaces may still not fit: GG_ENOMEM, nothing launched
            plan64.zeldovich(seed=1, out=out64)
            torch.cuda.synchronize()
        except gg.GGError as ex:
            out64, why = None, str(ex)
    else:
        why = "FP64 pos + vel grids (%.0f GB) do not fit in device memory" % (need / 1e9)
    if out64 is not None:
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            plan64.zeldovich(seed=1 + i, out=out64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / steps
        v64 = cells / (ms64 * 1e-3)
        fp64 = {"value": v64, "unit": "cells/s", "ms_per_step": ms64, "steps": steps,
                "fp32_speedup": value_per_gpu / v64}
        del out64
    else:
        fp64 = {"skipped": why}
    plan64.close()
    del plan64
    torch.cuda.empty_cache()
    return err, fp64


def main():
    args = parse()
    if args.workload == "batched_48" and args.impl == "ours":
        run_batched(args)
        return
    if args.workload.startswith("refine_"):
        run_refine(args)
        return
    if args.workload == "features_512":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "features_512 has no oracle arm; "
                              "the oracle is timed by the main workloads"}), flush=True)
            return
        run_features(args)
        return
    from paper_2511_10353_gb300.workloads import WORKLOADS
    w = dict(WORKLOADS[args.workload])
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    import paper_2511_10353_gb300 as gg
    from paper_2511_10353_gb300 import build
    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    else:
        dist = None
        torch.cuda.set_device(0)
    if rank == 0:
        build.build(verbose=False)
    if dist:
        dist.barrier()

    def barrier():
        if dist:
            dist.barrier()

    def allreduce_max(x):
        if not dist:
            return x
        tt = torch.tensor([x], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        return float(tt.item())

    dev_props = torch.cuda.get_device_properties(torch.cuda.current_device())
    gpu_id = "GPU-" + str(dev_props.uuid) if getattr(dev_props, "uuid", None) else str(local_rank)
    n = w["n"]
    cells = n ** 3
    res, plan, variants = time_plain(gg, w, args.steps, args.warmup, args.variants, world,
                                     barrier, gpu_id, allreduce_max, args.layout)
    chunked = res["config"]["spectrum_layout"] == "chunk-major"
    value = res["value"]
    line = {"metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if w["prec"] == "f32" else "f64", "data": "synthetic"}
    line.update({k: res[k] for k in ("config", "roofline", "path", "kernels", "gpu_launches",
                                     "clocks")})

    # FP64 plain path on the same workload, and the FP32 error against it
    if not args.no_fp64 and w["prec"] == "f32":
        k64 = max(2, min(10, args.steps // 10))
        line["err_vs_fp64"], line["fp64"] = fp64_leg(gg, w, plan, value / world, k64)
        plan = None

    # end to end through the public API with host buffers: caller white noise
    # (the paper's "WN from file" input) up, positions and velocities down
    if not args.no_e2e:
        dt = torch.float32 if w["prec"] == "f32" else torch.float64
        shape = (n, n, n)
        if plan is None:
            plan = gg.Plan(n, w["box"], w["cosmo"], w["z_init"], w["prec"])
            plan.set_variants(variants)
            plan.set_layout(chunked)
        hn = torch.randn(shape, dtype=dt).pin_memory()
        hout = {"psi": [None] * 3,
                "pos": [torch.empty(shape, dtype=dt, pin_memory=True) for _ in range(3)],
                "vel": [torch.empty(shape, dtype=dt, pin_memory=True) for _ in range(3)]}
        ke = max(5, min(10, args.steps // 4))
        plan.zeldovich_host(noise=hn, out=hout)
        barrier()
        t = time.perf_counter()
        for i in range(ke):
            plan.zeldovich_host(noise=hn, out=hout)
        el = allreduce_max(time.perf_counter() - t)
        esz = torch.finfo(dt).bits // 8
        # the copy engines' rates on the same pinned buffers, for scale: the
        # step's outputs are written by the kernels themselves over the host
        # link (mapped memory), which can beat the copies of a large buffer
        dev = torch.empty(shape, dtype=dt, device="cuda")
        rates = {}
        for name, fn in (("d2h", lambda: hout["pos"][0].copy_(dev, non_blocking=True)),
                         ("h2d", lambda: dev.copy_(hn, non_blocking=True))):
            fn()
            torch.cuda.synchronize()
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record()
            for _ in range(3):
                fn()
            c1.record()
            torch.cuda.synchronize()
            rates[name] = cells * esz * 3 / (c0.elapsed_time(c1) * 1e-3) / 1e9
        del dev
        bound_s = cells * esz / (rates["h2d"] * 1e9) + 6 * cells * esz / (rates["d2h"] * 1e9)
        line["e2e"] = {"value": world * cells * ke / el, "unit": "cells/s", "steps": ke,
                       "h2d_bytes_per_step": cells * esz, "d2h_bytes_per_step": 6 * cells * esz,
                       "api": "gg_zeldovich_host (pinned host noise in, pos/vel out)",
                       "timing": "host wall clock over the steps (each call synchronous)",
                       "copy_GB_s": rates, "copy_time_over_step_time": bound_s / (el / ke)}
        del hn, hout
    if plan is not None:
        plan.close()
        plan = None
    torch.cuda.empty_cache()

    # the 1536^3 precision workload (EH no-wiggle, 2000 Mpc/h), timed in the
    # same run when the headline workload is the default 512^3 one
    if args.workload == "zeldovich_512_fp32" and not args.no_1536:
        w2 = dict(WORKLOADS["zeldovich_1536_fp32"])
        k2 = max(10, min(20, args.steps))
        res2, plan2, _ = time_plain(gg, w2, k2, min(args.warmup, 3), None, world, barrier,
                                    gpu_id, allreduce_max)
        ns = {"workload": "zeldovich_1536_fp32", "unit": "cells/s"}
        ns.update(res2)
        if not args.no_fp64:
            ns["err_vs_fp64"], ns["fp64"] = fp64_leg(gg, w2, plan2, res2["value"] / world, 2)
        else:
            plan2.close()
        del plan2
        torch.cuda.empty_cache()
        line["zeldovich_1536_fp32"] = ns
        line["gpu_launches"] += res2["gpu_launches"]

    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, n_s=min(n, 512))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
