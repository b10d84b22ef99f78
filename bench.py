"""Throughput benchmark of the lightcone energy path.

One step = one evaluation of the batched energy workload: every edge
lightcone of a seeded random 3-regular graph (N = 100, p = 4, 150 edges)
for 64 angle sets, complex64 with FP64 edge products and energy sums, one
persistent launch (plus the angle-table, leaf-factor and energy kernels).
The metric is edge <Z_j Z_k> evaluations per second (edges x angle sets per
step / step time).

Multi-GPU (torchrun, one rank per GPU): edge x angle-set units are
independent, so every rank evaluates its own 64 angle sets of the same
graph (weak scaling) with no collective on the data path; only the step time
is reduced (max over ranks).

``--impl reference`` times the CPU FP64 oracle on a bounded sample of the
same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

METRIC = "edge ⟨ZZ⟩ evals/sec + energy-grad evals/sec on 1 GB300; % HBM/tensor roofline"
WORKLOAD = dict(name="n100_p4", batch=64, dtype="c64", order_trials=100)


# DRAM traffic of one persistent-kernel launch on the 100-vertex p = 4 graph,
# per angle set: dram__bytes_read.sum + dram__bytes_write.sum of one ncu
# capture at B = 4 angle sets, which grows in proportion to B (checked at
# B = 2), scaled to the launch's B.  It holds only for the kernel sources with
# this digest, for the plan with these algorithmic bytes per angle set (the
# contraction order fixes the traffic) and for this queue order (which sets
# what shares L2): otherwise the traffic is reported as null until that kernel
# and plan are captured again.
TRAFFIC_CAPTURES = [
    # orders searched per edge (100 trials), the bench plan; the queue takes the longest
    # remaining dependency path first (the default); fixed-fan-in row tile, task records
    # carrying dependency lists (profiles/persistent_kernel_n100p4_b4_dram.md).
    {"sources_sha256_16": "eccc125112799279", "alg_bytes_per_angle_set": 5170666432 / 4,
     "queue_order": "critical_path", "bytes_per_angle_set": (2322033664 + 2500920320) / 4},
    # the same after the warp-per-angle table search and the float-pair two-chunk tile
    {"sources_sha256_16": "cd11e675aaf9e03a", "alg_bytes_per_angle_set": 5170666432 / 4,
     "queue_order": "critical_path", "bytes_per_angle_set": (2330160896 + 2504982528) / 4},
]


def _kernel_digest():
    """Digest of the kernel sources as written (the key of the earlier captures)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("kernels.cu", "kernels.cuh", "qt_device.h"):
        h.update((ROOT / "paper_2106_15740_gb300" / "csrc" / f).read_bytes())
    return h.hexdigest()[:16]


def kernel_code_digest(texts=None):
    """Digest of the kernel sources' code: comments removed and runs of
    white space folded, so that a change to a comment keeps a capture valid
    and any change to the code voids it.  `texts` (the three files' contents)
    defaults to the files in the tree."""
    import hashlib
    import re
    if texts is None:
        texts = [(ROOT / "paper_2106_15740_gb300" / "csrc" / f).read_text()
                 for f in ("kernels.cu", "kernels.cuh", "qt_device.h")]
    h = hashlib.sha256()
    for t in texts:
        t = re.sub(r"/\*.*?\*/", " ", t, flags=re.S)
        t = re.sub(r"//[^\n]*", " ", t)
        h.update(" ".join(t.split()).encode())
    return h.hexdigest()[:16]


# Captures of the chained-step plan (which needs 34 or more angle sets, so a
# B = 4 capture does not have its steps) are taken on two edge ranges of the
# bench graph at B = 64 and give DRAM bytes per algorithmic byte; the two
# ranges agree when traffic grows in proportion to the plan's bytes, and the
# full launch's traffic is that ratio times its algorithmic bytes.
TRAFFIC_RATIO_CAPTURES = [
    # orders searched per edge (100 trials), chained steps of up to three consumers, the
    # longest-path queue; edges 40-80 and 0-40 at B = 64 (profiles/persistent_kernel_n100p4_b64_dram.md)
    {"sources_sha256_16": "615f58709fc2a191", "queue_order": "critical_path", "batch": 64, "fuse_chains": 3,
     "dram_bytes_per_alg_byte": (4694877696 + 5017392896 + 5532984320 + 5726372864) / (8730376192 + 9919264768)},
    # the same with the simulated list-scheduling queue order (the default)
    {"sources_sha256_16": "615f58709fc2a191", "queue_order": "simulated", "batch": 64, "fuse_chains": 3,
     "dram_bytes_per_alg_byte": (4737643264 + 5048140544 + 5629047040 + 5748539136) / (8730376192 + 9919264768)},
    # chains only from fan-in 2-3 buckets on the row-wide layout, multi-row tiles (per stored byte);
    # the simulated order with 9728 resident warps
    {"sources_sha256_16": "d95d15ebce694c8c", "queue_order": "simulated", "batch": 64, "fuse_chains": 3,
     "dram_bytes_per_alg_byte": (5102270464 + 5209602304 + 5970159360 + 5941778688) / (9256767488 + 10513176576)},
    # the same complex64 kernels after float-pair gradients (FP64 adjoints) were added to the sources
    # (digest of the code, comments ignored; as written: 5adb50b0ff9645eb)
    {"code_sha256_16": "9a5899f7577062f1", "queue_order": "simulated", "batch": 64, "fuse_chains": 3,
     "dram_bytes_per_alg_byte": (5105731840 + 5212003328 + 5965799424 + 5942155264) / (9256767488 + 10513176576)},
    # the same complex64 kernels after float-pair gradients took the multi-row tiles (2 to 16 angle sets)
    {"code_sha256_16": "f4d00e26317c1a4e", "queue_order": "simulated", "batch": 64, "fuse_chains": 3,
     "dram_bytes_per_alg_byte": (5089897984 + 5210417408 + 5966610432 + 5941371648) / (9256767488 + 10513176576)},
]


def _traffic(B, alg_bytes, profile_only):
    if profile_only:
        return None
    digest, code = _kernel_digest(), kernel_code_digest()
    order = WORKLOAD.get("queue_order", "simulated")
    for cap in TRAFFIC_CAPTURES:
        if (cap["sources_sha256_16"] == digest and cap["queue_order"] == order
                and abs(alg_bytes / B / cap["alg_bytes_per_angle_set"] - 1) < 1e-9):
            return cap["bytes_per_angle_set"] * B
    for cap in TRAFFIC_RATIO_CAPTURES:
        if ((cap.get("sources_sha256_16") == digest or cap.get("code_sha256_16") == code)
                and cap["queue_order"] == order and cap["batch"] == B
                and cap["fuse_chains"] == WORKLOAD.get("fuse_chains", 3)):
            return cap["dram_bytes_per_alg_byte"] * alg_bytes
    return None


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------- CPU oracle --

def _oracle_eval(args):
    name, edge, k = args
    from oracle import lightcone as lc
    from workloads import workload
    n, edges, p, g, b = workload(name, batch=WORKLOAD["batch"])
    v, _ = lc.lightcone_zz(n, edges, p, g[k], b[k], edge)
    return v.real


def _oracle_sample(n_items, seed):
    import numpy as np
    rng = np.random.default_rng(seed)
    return [(WORKLOAD["name"], int(e), int(k)) for e, k in zip(rng.integers(0, 150, n_items),
                                                               rng.integers(0, WORKLOAD["batch"], n_items))]


def _oracle_pool():
    import multiprocessing as mp
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    cores = min(os.cpu_count() or 1, 16)
    return mp.get_context("spawn").Pool(cores), cores


ERROR_ANGLE_SETS = (0, 21, 42, 63)


def cpu_baseline(budget_s=12.0, gpu_zz=None, gpu_e=None):
    """The oracle on host cores over a bounded sample of the workload.  With
    the GPU's per-edge values gpu_zz[edge, angle set] (real parts) and
    energies gpu_e[angle set] it also returns the errors against the oracle
    on every edge of ERROR_ANGLE_SETS: the largest per-edge |d<ZZ>| and the
    full-graph |dE| of each of those angle sets."""
    pool, cores = _oracle_pool()
    err = None
    try:
        pool.map(_oracle_eval, _oracle_sample(cores, 1))  # warm the workers
        if gpu_zz is not None:
            n_edges = gpu_zz.shape[0]
            chk = [(WORKLOAD["name"], e, k) for k in ERROR_ANGLE_SETS for e in range(n_edges)]
            vals = pool.map(_oracle_eval, chk, chunksize=8)
            ref = {(e, k): v for (_, e, k), v in zip(chk, vals)}
            d_e = {k: float(gpu_e[k]) - sum(0.5 * (1.0 - ref[(e, k)]) for e in range(n_edges)) for k in ERROR_ANGLE_SETS}
            err = {"pairs": len(chk),
                   "max_abs_dzz": max(abs(float(gpu_zz[e, k]) - v) for (e, k), v in ref.items()),
                   "abs_dE": {str(k): abs(v) for k, v in d_e.items()},
                   "max_abs_dE": max(abs(v) for v in d_e.values()),
                   "what": "complex64 bench path (the timed plan) vs the FP64 oracle: every edge of angle sets "
                           + ", ".join(map(str, ERROR_ANGLE_SETS)) + "; E over all 150 edges"}
        n_items = cores * 6
        t0 = time.perf_counter()
        done = 0
        while time.perf_counter() - t0 < budget_s:
            pool.map(_oracle_eval, _oracle_sample(n_items, 2 + done))
            done += n_items
        dt = time.perf_counter() - t0
        # one worker at a time: the single-thread rate on the same kind of sample
        t1 = time.perf_counter()
        single = 0
        for item in _oracle_sample(max(cores * 2, 8), 999):
            pool.apply(_oracle_eval, (item,))
            single += 1
            if time.perf_counter() - t1 > budget_s / 4:
                break
        dt1 = time.perf_counter() - t1
    finally:
        pool.terminate()
    return {"value": done / dt, "unit": "edge_evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} seeded (edge, angle-set) pairs of the N=100 p=4 workload, "
                      f"FP64 naive bucket elimination, {cores} worker processes x 1 thread",
            "single_thread": {"value": single / dt1, "unit": "edge_evals/s",
                              "sample": f"{single} pairs, one worker process x 1 thread"}}, err


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pool, cores = _oracle_pool()
    per_step = cores * 2
    try:
        for w in range(args.warmup):
            pool.map(_oracle_eval, _oracle_sample(per_step, 100 + w))
        t0 = time.perf_counter()
        for s in range(args.steps):
            pool.map(_oracle_eval, _oracle_sample(per_step, 200 + s))
        dt = time.perf_counter() - t0
    finally:
        pool.terminate()
    value = per_step * args.steps / dt
    sample = f"{per_step} seeded (edge, angle-set) pairs per step, FP64 oracle, {cores} processes"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "edge_evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "random 3-regular N=100 p=4, 150 edge lightcones x 64 angle sets (sampled)",
                   "graph_seed": 2, "angle_seed": 1002},
        "cpu_baseline": {"value": value, "unit": "edge_evals/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "edge_evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# -------------------------------------------------------------------- GPU --

class ClockSampler:
    def __init__(self, index, path):
        self.proc = None
        self.path = path
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={index}",
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in Path(self.path).read_text().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _time_calls(plan, g, b, grad, reps, torch, kernel=False):
    """Mean device time (ms) of `reps` plan evaluations after two warm-ups;
    with kernel=True also the mean time of the persistent bucket launch
    alone (the library's events around it, on the launching stream)."""
    from paper_2106_15740_gb300 import binding as qb
    for _ in range(2):
        plan.energy(g, b, grad=grad)
    plan.check()
    if kernel:
        qb.qt_plan_set_profiling(plan.plan, True)
        qb.qt_plan_kernel_times(plan.plan)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        plan.energy(g, b, grad=grad)
    t1.record()
    torch.cuda.synchronize()
    plan.check()
    ms = t0.elapsed_time(t1) / reps
    if not kernel:
        return ms
    k = qb.qt_plan_kernel_times(plan.plan)
    qb.qt_plan_set_profiling(plan.plan, False)
    return ms, sum(k) / max(1, len(k))


def _roofline(alg_bytes, kernel_ms, peak, peak_kind, kernel, stored_bytes=None):
    """Roofline of one launch: algorithmic bytes counted bucket by bucket
    (every bucket's intermediate inputs and result, the plan's per-unit figure
    times its units) over the kernel time.  A plan with chained steps stores
    and reads fewer bytes (`stored_bytes`), reported beside it."""
    achieved = alg_bytes / (kernel_ms * 1e-3) / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "kernel": kernel, "kernel_ms": kernel_ms, "alg_bytes_per_launch": alg_bytes, "peak_kind": peak_kind}
    if stored_bytes is not None and stored_bytes != alg_bytes:
        out["stored_bytes_per_launch"] = stored_bytes
        out["frac_of_stored_bytes"] = stored_bytes / (kernel_ms * 1e-3) / 1e9 / peak
        out["alg_bytes_what"] = ("bucket by bucket: every bucket's intermediate inputs and result; the chained "
                                 "steps keep the results of the buckets they absorb in registers, so the launch "
                                 "stores and reads stored_bytes_per_launch")
    return out


# This GPU's FP64 rate (nominal, dense, the same on the FP64 units and the
# tensor pipe): 1.25 TFLOP/s, about 2 FP64 fused multiply-adds per SM per clock
# at 152 SMs and 2.07 GHz.
FP64_TFLOPS_NOMINAL = 1.25


def _roofline_fp64(flops, kernel_ms):
    """ALU roofline of a complex128 launch: the plan's real FLOPs (per bucket
    6 (k - 1) 2^|U| for the products of its k inputs at both values of the
    eliminated variable, plus 2^|U| for the sum over it, times the angle sets)
    over the kernel time, against the nominal FP64 rate.  One complex product
    is 6 FLOPs in 4 FP64 instructions (2 multiplies, 2 fused multiply-adds), so
    a kernel that keeps the FP64 units busy with nothing else reaches about
    0.72 of the nominal rate by this count."""
    achieved = flops / (kernel_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP64_TFLOPS_NOMINAL, "unit": "TFLOP/s",
            "frac": achieved / FP64_TFLOPS_NOMINAL, "peak_kind": "nominal FP64 rate (dense)",
            "flops_per_launch": flops, "kernel_ms": kernel_ms}


def min_fill_comparison(n, edges, p, B, g, b, dev, torch):
    """The same step with the plain greedy min-fill order (more bytes)."""
    from paper_2106_15740_gb300.energy import EnergyPlan
    plan = EnergyPlan(n, edges, p, batch=B, dtype=WORKLOAD["dtype"], mode="persistent", device=dev)
    ms = _time_calls(plan, g, b, False, 5, torch)
    out = {"value": len(edges) * B / (ms * 1e-3), "unit": "edge_evals/s", "ms_per_step": ms,
           "alg_bytes_per_step": plan.stats["alg_bytes"], "max_width": int(plan.stats["max_width"]),
           "achieved_gbs": plan.stats["alg_bytes"] / (ms * 1e-3) / 1e9}
    plan.close()
    return out


def _plan_variant(n, edges, p, B, g, b, dev, torch, what, **kw):
    """The bench step's plan and tile with one planning option changed (direct calls)."""
    from paper_2106_15740_gb300.energy import EnergyPlan
    plan = EnergyPlan(n, edges, p, batch=B, dtype=WORKLOAD["dtype"], mode="persistent", device=dev,
                      order_trials=WORKLOAD.get("order_trials", 0), lane_items=WORKLOAD.get("lane_items", 0),
                      group_rows=WORKLOAD.get("group_rows", 0), **kw)
    ms, kms = _time_calls(plan, g, b, False, 5, torch, kernel=True)
    peak, peak_kind = _peaks()
    alg = plan.bucket_bytes()
    out = {"value": len(edges) * B / (ms * 1e-3), "unit": "edge_evals/s", "ms_per_step": ms,
           "alg_bytes_per_step": alg, "stored_bytes_per_step": plan.stats["alg_bytes"],
           "achieved_gbs": alg / (ms * 1e-3) / 1e9, "what": what,
           "roofline": _roofline(alg, kms, peak, peak_kind, "persistent_kernel", plan.stats["alg_bytes"])}
    plan.close()
    torch.cuda.empty_cache()
    return out


def chain_comparison(n, edges, p, B, g, b, dev, torch):
    """The bench step with every step of a workspace slot chained to the one
    before it (chain_steps), instead of waiting only for its tree dependencies."""
    return _plan_variant(n, edges, p, B, g, b, dev, torch,
                         "same plan and tile, each step waits for the step before it on its slot (direct calls)",
                         chain_steps=True)


def round_robin_comparison(n, edges, p, B, g, b, dev, torch):
    """The bench step with the queue taken round-robin over the workspace
    slots, step by step, instead of the simulated list-scheduling order."""
    return _plan_variant(n, edges, p, B, g, b, dev, torch,
                         "same plan and tile, queue round-robin over slots step by step (direct calls)",
                         queue_order="round_robin")


def critical_path_comparison(n, edges, p, B, g, b, dev, torch):
    """The bench step with the queue sorted by longest remaining dependency
    path alone (no simulation of the warps)."""
    return _plan_variant(n, edges, p, B, g, b, dev, torch,
                         "same plan and tile, queue sorted by longest remaining path (direct calls)",
                         queue_order="critical_path")


def unfused_comparison(n, edges, p, B, g, b, dev, torch):
    """The bench step with every bucket a step of its own (fuse_chains off):
    each chained bucket's result is written and read back."""
    return _plan_variant(n, edges, p, B, g, b, dev, torch,
                         "same orders and tile, every bucket a step of its own (no chained steps; direct calls)",
                         fuse_chains=False)


def gradient_and_comparator(dev, torch):
    """Energy-gradient throughput on the 60-vertex p = 4 workload (8 angles,
    one angle set, adjoint sweep) in complex64, complex128 and float pairs, and the plain
    per-edge complex128 contraction (one kernel launch per bucket, edge after
    edge, one angle set at a time) on the gradient workload and on the bench
    workload (all 64 angle sets of one bench step, measured)."""
    from paper_2106_15740_gb300.energy import EnergyPlan
    from workloads import random_angles, workload
    peak, peak_kind = _peaks()
    out = {}
    n, edges, p, g, b = workload("n60_p4")
    gd, bd = torch.tensor(g, device=dev), torch.tensor(b, device=dev)
    # tile size, grouping and per-width schedule of the gradient plan, picked on this device
    from paper_2106_15740_gb300.energy import autotune, autotune_bands
    trials = WORKLOAD.get("order_trials", 0)
    best, timings = autotune(n, edges, p, batch=1, dtype="c64", gradient=True, device=dev, reps=3,
                             lane_items=(16, 32, 64), group_rows=(0, 32), order_trials=trials)
    by_rank, band_ms = autotune_bands(n, edges, p, batch=1, dtype="c64", gradient=True, device=dev, reps=3,
                                      order_trials=trials, **best)
    tuned = dict(best, chunk_tiles_by_rank=by_rank)
    res = {}
    for dt in ("c64", "c128", "c64x2"):
        plan = EnergyPlan(n, edges, p, batch=1, dtype=dt, mode="persistent", gradient=True, device=dev,
                          order_trials=trials, **tuned)
        ms, kms = _time_calls(plan, gd, bd, True, 5, torch, kernel=True)
        _, gr = plan.energy(gd, bd, grad=True)
        res[dt] = dict(ms=ms, kms=kms, alg=plan.stats["alg_bytes"], grad=gr.cpu().numpy()[0])
        plan.close()
    plan = EnergyPlan(n, edges, p, batch=1, dtype="c64", mode="persistent", gradient=True, device=dev)
    ms_grad_mf = _time_calls(plan, gd, bd, True, 3, torch)
    plan.close()
    plan = EnergyPlan(n, edges, p, batch=1, dtype="c128", mode="per_bucket", device=dev)
    ms_loop = _time_calls(plan, gd, bd, False, 3, torch)
    plan.close()
    gb, bb = random_angles(16, p, 1003)
    plan = EnergyPlan(n, edges, p, batch=16, dtype="c64", mode="persistent", gradient=True, device=dev,
                      order_trials=WORKLOAD.get("order_trials", 0))
    ms_grad16 = _time_calls(plan, torch.tensor(gb, device=dev), torch.tensor(bb, device=dev), True, 3, torch)
    plan.close()
    c64, c128, c64x2 = res["c64"], res["c128"], res["c64x2"]
    out["grad"] = {"metric": "energy-grad evals/sec", "value": 1e3 / c64["ms"], "unit": "grad_evals/s",
                   "batched_16": {"value": 16e3 / ms_grad16, "ms_per_call": ms_grad16,
                                  "what": "16 angle sets per call (a multi-start optimiser's batch)"},
                   "ms_per_eval": c64["ms"], "dtype": "c64",
                   "workload": "random 3-regular N=60 p=4 (seed 3), 90 edge lightcones, dE/dgamma and dE/dbeta "
                               "(8 angles) by the adjoint bucket sweep, one angle set",
                   "ordering": f"searched, {WORKLOAD.get('order_trials', 0)} trials per edge",
                   "autotune": {"choice": best, "per_width_band": band_ms,
                                "ms_per_candidate": {f"lane_items={k[0]},group_rows={k[1]}": round(v, 3)
                                                     for k, v in timings.items()}},
                   "alg_bytes_per_eval": c64["alg"], "achieved_gbs": c64["alg"] / (c64["ms"] * 1e-3) / 1e9,
                   "roofline": _roofline(c64["alg"], c64["kms"], peak, peak_kind,
                                         "persistent_kernel<float,1,true,true,2>"),
                   "c128": {"value": 1e3 / c128["ms"], "ms_per_eval": c128["ms"], "alg_bytes_per_eval": c128["alg"],
                            "roofline": _roofline(c128["alg"], c128["kms"], peak, peak_kind,
                                                  "persistent_kernel<double,1,true,true,2>")},
                   "c64x2": {"value": 1e3 / c64x2["ms"], "ms_per_eval": c64x2["ms"],
                             "alg_bytes_per_eval": c64x2["alg"],
                             "roofline": _roofline(c64x2["alg"], c64x2["kms"], peak, peak_kind,
                                                   "persistent_kernel<ff,1,true,true,2> (float pairs)"),
                             "max_abs_dgrad_vs_c128": float(abs(c64x2["grad"] - c128["grad"]).max())},
                   "max_abs_dgrad_c64_vs_c128": float(abs(c64["grad"] - c128["grad"]).max()),
                   "max_abs_grad": float(abs(c128["grad"]).max()),
                   "min_fill_order_ms_per_eval": ms_grad_mf,
                   "per_edge_c128_forward_ms": ms_loop,
                   "speedup_vs_per_edge_c128_forward": ms_loop / c64["ms"]}
    n, edges, p, g, b = workload("n100_p4", batch=64)
    plan = EnergyPlan(n, edges, p, batch=1, dtype="c128", mode="per_bucket", device=dev)
    gs = [torch.tensor(g[k:k + 1], device=dev) for k in range(64)]
    bs = [torch.tensor(b[k:k + 1], device=dev) for k in range(64)]
    plan.energy(gs[0], bs[0])
    plan.check()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for k in range(64):
        plan.energy(gs[k], bs[k])
    t1.record()
    torch.cuda.synchronize()
    plan.check()
    ms_step = t0.elapsed_time(t1)
    plan.close()
    out["per_edge_c128_loop"] = {"ms_per_step": ms_step, "ms_per_angle_set": ms_step / 64,
                                 "edge_evals_per_s": 64 * len(edges) / (ms_step * 1e-3),
                                 "what": "same graph, complex128, one launch per bucket, edges one after "
                                         "another, one angle set per call: all 64 calls of one bench step, measured"}
    return out


def complex128_counterparts(dev, torch):
    """The bench plan (150 edges x 64 angle sets, searched orders, one
    persistent launch) in complex128 and in float pairs (c64x2), and the
    100-vertex p = 3 graph (one angle set) in the three precisions: time,
    roofline, and the complex64 and float-pair errors against complex128."""
    import numpy as np
    from paper_2106_15740_gb300.energy import EnergyPlan
    from workloads import workload
    peak, peak_kind = _peaks()
    out = {}
    for name, B, trials in (("n100_p4", 64, WORKLOAD.get("order_trials", 0)), ("n100_p3", 1, 0)):
        n, edges, p, g, b = workload(name, batch=B)
        gd, bd = torch.tensor(g, device=dev), torch.tensor(b, device=dev)
        r = {}
        for dt in ("c64", "c128", "c64x2"):
            plan = EnergyPlan(n, edges, p, batch=B, dtype=dt, mode="persistent", device=dev, order_trials=trials)
            ms, kms = _time_calls(plan, gd, bd, False, 5, torch, kernel=True)
            e, zz = plan.energy(gd, bd, edge_zz=True)
            plan.check()
            r[dt] = dict(ms=ms, kms=kms, alg=plan.bucket_bytes(), stored=plan.stats["alg_bytes"],
                         flops=plan.stats["flops"], e=e.cpu().numpy(), zz=zz.cpu().numpy())
            plan.close()
        key = "n100_p4_b64" if B == 64 else "n100_p3_b1"
        out[key] = {
            "c128": {"value": len(edges) * B / (r["c128"]["ms"] * 1e-3), "unit": "edge_evals/s",
                     "ms_per_call": r["c128"]["ms"],
                     "roofline": _roofline(r["c128"]["alg"], r["c128"]["kms"], peak, peak_kind, "persistent_kernel<double,...>",
                                           r["c128"]["stored"]),
                     "roofline_fp64": _roofline_fp64(r["c128"]["flops"], r["c128"]["kms"])},
            "c64": {"value": len(edges) * B / (r["c64"]["ms"] * 1e-3), "unit": "edge_evals/s",
                    "ms_per_call": r["c64"]["ms"],
                    "roofline": _roofline(r["c64"]["alg"], r["c64"]["kms"], peak, peak_kind, "persistent_kernel<float,...>",
                                           r["c64"]["stored"])},
            "c64x2": {"value": len(edges) * B / (r["c64x2"]["ms"] * 1e-3), "unit": "edge_evals/s",
                      "ms_per_call": r["c64x2"]["ms"],
                      "roofline": _roofline(r["c64x2"]["alg"], r["c64x2"]["kms"], peak, peak_kind,
                                            "persistent_kernel<ff,...> (float pairs)", r["c64x2"]["stored"])},
            "c64_vs_c128": {"max_abs_dzz": float(np.abs(r["c64"]["zz"][:, :, 0] - r["c128"]["zz"][:, :, 0]).max()),
                            "max_abs_dE": float(np.abs(r["c64"]["e"] - r["c128"]["e"]).max())},
            "c64x2_vs_c128": {"max_abs_dzz": float(np.abs(r["c64x2"]["zz"][:, :, 0] - r["c128"]["zz"][:, :, 0]).max()),
                              "max_abs_dE": float(np.abs(r["c64x2"]["e"] - r["c128"]["e"]).max())},
            "workload": f"{name}, {len(edges)} edges x {B} angle sets, "
                        + (f"searched orders ({trials} trials)" if trials else "min-fill orders")}
    return out


def large_config(dev, torch):
    """The 244-vertex p = 5 graph (366 edges): searched orders (100 trials),
    width budget 28 with slicing; energy and energy + gradient in complex64,
    energy in complex128 for the error; one angle set."""
    import numpy as np
    from paper_2106_15740_gb300.energy import EnergyPlan
    from workloads import workload
    peak, peak_kind = _peaks()
    n, edges, p, g, b = workload("n244_p5")
    gd, bd = torch.tensor(g, device=dev), torch.tensor(b, device=dev)
    kw = dict(batch=1, mode="persistent", device=dev, order_trials=100, max_width=28, slice=True,
              max_workspace=100 << 30)
    out = {"workload": "random 3-regular N=244 p=5 (seed 4), 366 edge lightcones, one angle set, searched orders "
                       "(100 trials), width budget 28 (wider edges sliced)"}
    plan = EnergyPlan(n, edges, p, dtype="c64", **kw)
    ms, kms = _time_calls(plan, gd, bd, False, 3, torch, kernel=True)
    e64, zz64 = plan.energy(gd, bd, edge_zz=True)
    plan.check()
    out["energy_c64"] = {"value": len(edges) / (ms * 1e-3), "unit": "edge_evals/s", "ms_per_call": ms,
                         "max_width": int(plan.widths.max()), "sliced_edges": int((plan.slices > 0).sum()),
                         "networks": int((2 ** plan.slices.astype(np.int64)).sum()),
                         "roofline": _roofline(plan.bucket_bytes(), kms, peak, peak_kind,
                                               "persistent_kernel<float,1,true,false,4>", plan.stats["alg_bytes"])}
    plan.close()
    torch.cuda.empty_cache()
    plan = EnergyPlan(n, edges, p, dtype="c64", fuse_chains=0, **kw)
    ms0, kms0 = _time_calls(plan, gd, bd, False, 2, torch, kernel=True)
    out["energy_c64_unfused"] = {"value": len(edges) / (ms0 * 1e-3), "unit": "edge_evals/s", "ms_per_call": ms0,
                                 "what": "the same plan with every bucket a step of its own (fuse_chains=0)",
                                 "roofline": _roofline(plan.stats["alg_bytes"], kms0, peak, peak_kind,
                                                       "persistent_kernel<float,1,true,false,2>")}
    plan.close()
    torch.cuda.empty_cache()
    plan = EnergyPlan(n, edges, p, dtype="c64", gradient=True, **kw)
    ms, kms = _time_calls(plan, gd, bd, True, 2, torch, kernel=True)
    _, g64 = plan.energy(gd, bd, grad=True)
    plan.check()
    out["energy_grad_c64"] = {"value": 1e3 / ms, "unit": "grad_evals/s", "ms_per_call": ms,
                              "roofline": _roofline(plan.stats["alg_bytes"], kms, peak, peak_kind,
                                                    "persistent_kernel<float,1,true,true,2>")}
    plan.close()
    torch.cuda.empty_cache()
    plan = EnergyPlan(n, edges, p, dtype="c64x2", **kw)
    msx2, kmsx2 = _time_calls(plan, gd, bd, False, 1, torch, kernel=True)
    ex2, zzx2 = plan.energy(gd, bd, edge_zz=True)
    plan.check()
    out["energy_c64x2"] = {"value": len(edges) / (msx2 * 1e-3), "unit": "edge_evals/s", "ms_per_call": msx2,
                           "roofline": _roofline(plan.bucket_bytes(), kmsx2, peak, peak_kind,
                                                 "persistent_kernel<ff,1,true,false,4> (float pairs)",
                                                 plan.stats["alg_bytes"])}
    plan.close()
    torch.cuda.empty_cache()
    plan = EnergyPlan(n, edges, p, dtype="c128", **kw)
    ms128 = _time_calls(plan, gd, bd, False, 1, torch)
    e128, zz128 = plan.energy(gd, bd, edge_zz=True)
    plan.check()
    plan.close()
    torch.cuda.empty_cache()
    out["energy_c128_ms_per_call"] = ms128
    out["c64_vs_c128"] = {"max_abs_dzz": float((zz64[:, 0, 0] - zz128[:, 0, 0]).abs().max()),
                          "abs_dE": float((e64 - e128).abs().max())}
    out["c64x2_vs_c128"] = {"max_abs_dzz": float((zzx2[:, 0, 0] - zz128[:, 0, 0]).abs().max()),
                            "abs_dE": float((ex2 - e128).abs().max())}
    return out


def amplitude_measure(dev, torch):
    """Single-amplitude cost on the paper's benchmark shape (§Results: one
    amplitude of the full circuit of a random 3-regular graph, 40 vertices,
    p = 3, the depth the paper reaches on a 4 GB laptop with ZZ and diagonal
    gates): 8 seeded bitstrings, one angle set, complex128 (the paper's
    precision), float pairs and complex64, searched orders."""
    import numpy as np
    from paper_2106_15740_gb300.amplitude import AmplitudePlan
    from workloads import random_angles, random_regular_graph
    n, p = 40, 3
    edges = random_regular_graph(n, 3, 0)
    g, b = random_angles(1, p, 1000)
    bits = np.random.default_rng(7).integers(0, 2, (8, n)).astype(np.uint8)
    gd, bd = torch.tensor(g, device=dev), torch.tensor(b, device=dev)
    out = {"workload": "random 3-regular N=40 p=3 (seed 0), 8 bitstrings x 1 angle set, full-circuit ket networks, "
                       "100 order trials per bitstring"}
    for dtype in ("c128", "c64x2", "c64"):
        plan = AmplitudePlan(n, edges, p, bits, batch=1, dtype=dtype, order_trials=100, device=dev)
        for _ in range(2):
            plan.amplitudes(gd, bd)
        plan.check()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(5):
            plan.amplitudes(gd, bd)
        t1.record()
        torch.cuda.synchronize()
        plan.check()
        ms = t0.elapsed_time(t1) / 5
        out[dtype] = {"amplitudes_per_s": 8 / (ms * 1e-3), "ms_per_call": ms, "max_width": int(max(plan.widths)),
                      "alg_bytes_per_call": plan.stats["alg_bytes"],
                      "achieved_gbs": plan.stats["alg_bytes"] / (ms * 1e-3) / 1e9}
        plan.close()
    return out


def run_ours(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_15740_gb300 import binding as qb
    from paper_2106_15740_gb300.energy import EnergyPlan
    from workloads import random_angles, workload

    n, edges, p, _, _ = workload(WORKLOAD["name"])
    B = WORKLOAD["batch"]
    profile_only = ((WORKLOAD["name"], B) != ("n100_p4", 64) or "edge_range" in WORKLOAD or "lane_items" in WORKLOAD
                    or "chunk_tiles" in WORKLOAD or "gradient" in WORKLOAD or "max_width" in WORKLOAD
                    or "profile_order" in WORKLOAD
                    or "chain_steps" in WORKLOAD or "queue_order" in WORKLOAD)
    grad = bool(WORKLOAD.get("gradient", False))
    gamma, beta = random_angles(B, p, 1002 + 7919 * rank)
    tuned = None
    if not profile_only:
        # tile size and grouping picked on this device, before the timed region
        from paper_2106_15740_gb300.energy import autotune
        best, timings = autotune(n, edges, p, batch=B, dtype=WORKLOAD["dtype"], device=dev, reps=3,
                                 lane_items=(16, 32, 64), group_rows=(0, -1, 32),
                                 order_trials=WORKLOAD.get("order_trials", 0))
        WORKLOAD["lane_items"], WORKLOAD["group_rows"] = best["lane_items"], best["group_rows"]
        # then the per-width schedule: warp tiles per queue task by band of output ranks
        from paper_2106_15740_gb300.energy import autotune_bands
        by_rank, band_ms = autotune_bands(n, edges, p, batch=B, dtype=WORKLOAD["dtype"], device=dev, reps=3,
                                          order_trials=WORKLOAD.get("order_trials", 0),
                                          lane_items=best["lane_items"], group_rows=best["group_rows"])
        WORKLOAD["chunk_tiles_by_rank"] = by_rank
        tuned = {"choice": best,
                 "ms_per_candidate": {f"lane_items={k[0]},group_rows={k[1]}": round(v, 3) for k, v in timings.items()},
                 "per_width_band": band_ms}
    t_plan = time.perf_counter()
    plan = EnergyPlan(n, edges, p, batch=B, dtype=WORKLOAD["dtype"], mode="persistent", device=dev,
                      edge_range=WORKLOAD.get("edge_range"), lane_items=WORKLOAD.get("lane_items", 0),
                      group_rows=WORKLOAD.get("group_rows", 0), chunk_tiles=WORKLOAD.get("chunk_tiles", 0),
                      gradient=grad, max_width=WORKLOAD.get("max_width", 0), slice=WORKLOAD.get("slice", False),
                      max_workspace=WORKLOAD.get("max_workspace", 0), order_trials=WORKLOAD.get("order_trials", 0),
                      chain_steps=WORKLOAD.get("chain_steps", False),
                      queue_order=WORKLOAD.get("queue_order", "simulated"),
                      chunk_tiles_by_rank=WORKLOAD.get("chunk_tiles_by_rank"))
    t_plan = time.perf_counter() - t_plan
    from paper_2106_15740_gb300.schedule import bytes_by_rank
    g = torch.tensor(gamma, device=dev)
    b = torch.tensor(beta, device=dev)
    out = torch.empty(B, dtype=torch.float64, device=dev)
    units = plan.n_edges * B

    # One step = one replay of the evaluation captured as a CUDA graph.
    step = plan.capture(grad=grad)
    step(g, b)
    for _ in range(args.warmup):
        step.replay()
    plan.check()

    stream = torch.cuda.current_stream(dev)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local, os.path.join(tempfile.gettempdir(), f"qt_bench_clocks_{os.getpid()}.csv")) \
        if rank == 0 else None
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    t0.record(stream)
    marks[0].record(stream)
    for i in range(args.steps):
        step.replay()
        marks[i + 1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    plan.check()
    ms = t0.elapsed_time(t1) / args.steps
    per_step = sorted(marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps))

    # Kernel time of the persistent launch: the same K steps as direct calls
    # with the library's profiling events around the bucket launch (events
    # on the launching stream), right after the graph-timed steps.
    qb.qt_plan_set_profiling(plan.plan, True)
    qb.qt_plan_kernel_times(plan.plan)
    t0.record(stream)
    for _ in range(args.steps):
        plan.energy(g, b, out=out, grad=grad)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop() if clocks else None
    plan.check()
    ms_direct = t0.elapsed_time(t1) / args.steps
    kernel_ms = qb.qt_plan_kernel_times(plan.plan)
    qb.qt_plan_set_profiling(plan.plan, False)
    if pg:
        t = torch.tensor([ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())

    # End to end through the public host-pointer call: angles H2D from pinned
    # host memory, energies D2H, every step.
    hg = torch.tensor(gamma).pin_memory().numpy()
    hb = torch.tensor(beta).pin_memory().numpy()
    for _ in range(2):
        plan.energy_host(hg, hb)
    if pg:
        pg.barrier()
    w0 = time.perf_counter()
    for _ in range(args.steps):
        plan.energy_host(hg, hb)
    e2e_s = (time.perf_counter() - w0) / args.steps
    if pg:
        t = torch.tensor([e2e_s], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        e2e_s = float(t.item())

    peak, peak_kind = _peaks()
    kms = sum(kernel_ms) / max(1, len(kernel_ms))
    stored = plan.stats["alg_bytes"]  # what the plan's steps store and read
    alg = plan.bucket_bytes()  # bucket by bucket (every bucket's inputs and result): the roofline's bytes
    achieved = alg / (kms * 1e-3) / 1e9
    if rank == 0:
        res = {
            "metric": METRIC, "value": units * world / (ms * 1e-3), "unit": "edge_evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": WORKLOAD["dtype"],
            "data": "synthetic",
            "config": {"workload": ("random 3-regular N=100 p=4 (seed 2), 150 edge lightcones x 64 angle sets, "
                                    "complex64 + FP64 sums, persistent launch") if not profile_only else
                                   f"profiling case {WORKLOAD}",
                       "ordering": (f"per edge the cheapest of greedy min-fill and {WORKLOAD.get('order_trials', 0)} "
                                    "seeded randomised greedy orders (seed 0, tau 1), no wider than min-fill"
                                    if WORKLOAD.get("order_trials", 0) else "greedy min-fill"),
                       "alg_bytes_per_step": alg, "stored_bytes_per_step": stored,
                       "n_vertices": n, "p": p, "edges": len(edges), "angle_sets_per_gpu": B,
                       "max_width": int(plan.stats["max_width"]), "buckets": plan.stats["n_buckets"],
                       "width_histogram": {int(w): int(c) for w, c in zip(*np.unique(plan.widths, return_counts=True))},
                       "workspace_gb": round(plan.ws_bytes / 1e9, 2),
                       "l2": "working set larger than L2 (intermediates streamed through HBM every step)",
                       "plan_host_s": round(t_plan, 3),
                       "alg_bytes_by_result_rank": bytes_by_rank(plan.plan, B, 8 if WORKLOAD["dtype"] == "c64" else 16)},
            "roofline": dict(_roofline(alg, kms, peak, peak_kind, "persistent_kernel<float,2,false,false,4>", stored),
                             traffic=_traffic(B, stored, profile_only),
                             kernel_ms_from="CUDA events around the persistent launch over K direct calls after "
                                            "the graph-timed steps"),
            "e2e": {"value": units * world / e2e_s, "unit": "edge_evals/s",
                    "h2d_bytes_per_step": int(2 * B * p * 8), "d2h_bytes_per_step": int(B * 8)},
            "gpu_launches": (7 if grad else 4) * args.steps,
            "step_form": {"timed": "K replays of one CUDA graph holding the evaluation "
                                   "(angle table, leaf factors, persistent launch, FP64 energy sum)",
                          "ms_per_step_direct_calls": ms_direct},
            "step_ms": {"mean": ms, "median": per_step[len(per_step) // 2], "min": per_step[0],
                        "max": per_step[-1], "steps": len(per_step),
                        "what": "CUDA events between consecutive graph replays of the timed region"},
            "clocks": clk,
        }
        if tuned:
            res["autotune"] = tuned
        if profile_only:
            res["profile_only"] = f"{WORKLOAD} (not the bench workload)"
        if not profile_only and WORKLOAD.get("order_trials", 0):
            res["min_fill_order"] = min_fill_comparison(n, edges, p, B, g, b, dev, torch)
        if not profile_only:
            res["chained_steps"] = chain_comparison(n, edges, p, B, g, b, dev, torch)
            res["round_robin_queue"] = round_robin_comparison(n, edges, p, B, g, b, dev, torch)
            res["critical_path_queue"] = critical_path_comparison(n, edges, p, B, g, b, dev, torch)
            res["unfused_chains"] = unfused_comparison(n, edges, p, B, g, b, dev, torch)
        if not args.no_cpu_baseline:
            e_gpu, zz = plan.energy(g, b, edge_zz=True)
            plan.check()
            zz_host, e_host = zz[:, :, 0].cpu().numpy(), e_gpu.cpu().numpy()
            plan.close()
            torch.cuda.empty_cache()
            res.update(gradient_and_comparator(dev, torch))
            res["complex128"] = complex128_counterparts(dev, torch)
            res["large"] = large_config(dev, torch)
            res["single_amplitude"] = amplitude_measure(dev, torch)
            res["per_edge_c128_loop"]["speedup_of_value"] = res["value"] / res["per_edge_c128_loop"]["edge_evals_per_s"]
            res["cpu_baseline"], res["error_vs_oracle"] = cpu_baseline(gpu_zz=zz_host, gpu_e=e_host)
        print(json.dumps(res))
    if pg:
        pg.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=None, help="profiling only: angle sets per GPU")
    ap.add_argument("--workload", default=None, help="profiling only: named workload of workloads.py")
    ap.add_argument("--dtype", default=None, choices=["c64", "c128", "c64x2"], help="profiling only")
    ap.add_argument("--edges", default=None, help="profiling only: edge range a:b of the graph")
    ap.add_argument("--lane-items", type=int, default=0, help="profiling only: warp tile items per lane")
    ap.add_argument("--group-rows", type=int, default=0, help="profiling only: grouping threshold")
    ap.add_argument("--chunk-tiles", type=int, default=0, help="profiling only: warp tiles per queue task")
    ap.add_argument("--gradient", action="store_true", help="profiling only: time the energy + adjoint gradient")
    ap.add_argument("--max-width", type=int, default=0, help="profiling only: width budget")
    ap.add_argument("--slice", action="store_true", help="profiling only: slice edges above the width budget")
    ap.add_argument("--max-workspace-gb", type=float, default=0, help="profiling only: workspace cap")
    ap.add_argument("--chain-steps", action="store_true",
                    help="profiling only: chain every step of a workspace slot to the one before it")
    ap.add_argument("--queue-order", default=None, choices=["round_robin", "critical_path", "simulated"],
                    help="profiling only: order of the persistent queue")
    ap.add_argument("--order-trials", type=int, default=None,
                    help="profiling only: randomised greedy orders per edge (0: min-fill)")
    args = ap.parse_args()
    if args.edges:
        a, b = (int(x) for x in args.edges.split(":"))
        WORKLOAD["edge_range"] = (a, b)
        args.no_cpu_baseline = True
    if args.lane_items or args.group_rows:
        WORKLOAD["lane_items"], WORKLOAD["group_rows"] = args.lane_items, args.group_rows
    if args.chunk_tiles:
        WORKLOAD["chunk_tiles"] = args.chunk_tiles
        args.no_cpu_baseline = True
    if args.gradient:
        WORKLOAD["gradient"] = True
        args.no_cpu_baseline = True
    if args.max_width:
        WORKLOAD["max_width"], WORKLOAD["slice"] = args.max_width, args.slice
        args.no_cpu_baseline = True
    if args.order_trials is not None:
        WORKLOAD["order_trials"] = args.order_trials
        WORKLOAD["profile_order"] = True
        args.no_cpu_baseline = True
    if args.chain_steps:
        WORKLOAD["chain_steps"] = True
        args.no_cpu_baseline = True
    if args.queue_order is not None:
        WORKLOAD["queue_order"] = args.queue_order
        args.no_cpu_baseline = True
    if args.max_workspace_gb:
        WORKLOAD["max_workspace"] = int(args.max_workspace_gb * (1 << 30))
    for key in ("batch", "workload", "dtype"):
        val = getattr(args, key)
        if val is not None:
            WORKLOAD["name" if key == "workload" else key] = val
            args.no_cpu_baseline = True
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
