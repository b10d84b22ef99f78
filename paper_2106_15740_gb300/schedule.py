"""Dependency statistics of a persistent plan's queue (host only, no device).

A persistent plan queues every step of every network in one launch; a step
waits for the steps on its dependency list (``qt_plan_schedule``).  This
module measures that graph: the number of queued units (a step's chunks, or
a group of tiny steps that one warp runs in order), the dependencies per
unit, and the longest dependency path in units, which bounds how many steps
one after another the launch must wait through.  With ``chain_steps`` every
step of a workspace slot waits for the one before it, so the path is the
length of a slot's step list.  ``trace_stats`` summarises a queue trace taken
on the device (``EnergyPlan.trace``): time working, waiting and idle, and the
start-up phase before all warps are busy.

    python -m paper_2106_15740_gb300.schedule      # the bench and gradient workloads
"""
from __future__ import annotations

import numpy as np

from . import binding as qb


def schedule_stats(plan) -> dict:
    """{"units", "tasks", "deps_per_unit", "max_deps", "longest_path"} of a
    persistent plan handle (``qt_plan_create``)."""
    sch = qb.qt_plan_schedule(plan)
    tasks = qb.qt_plan_tasks(plan)
    unit = sch["unit"]
    depth = {}
    order = []
    seen = set()
    for s in tasks["step"]:  # units in queue order: every dependency comes earlier
        s = int(s)
        if s not in seen:
            seen.add(s)
            order.append(s)
    for u in order:
        d0, dc = int(sch["dep_first"][u]), int(sch["dep_count"][u])
        depth[u] = 1 + max((depth[int(unit[d])] for d in sch["deps"][d0:d0 + dc]), default=0)
    n_units = len(order)
    return {"units": n_units, "tasks": int(len(tasks["step"])),
            "deps_per_unit": float(len(sch["deps"])) / max(n_units, 1),
            "max_deps": int(sch["dep_count"].max()) if n_units else 0,
            "longest_path": max(depth.values()) if depth else 0}


def bytes_by_rank(plan, batch, elem_bytes, threshold=18) -> dict:
    """Algorithmic bytes of a persistent plan split by the steps' result rank:
    steps whose output has rank >= threshold stream their operands through
    HBM; narrower ones work mostly out of L2.  A step's bytes are the
    elements it reads and writes (its intermediate inputs and its output;
    leaf factors are not counted) times elem_bytes, so that over all steps
    they sum to the plan's algorithmic bytes (gradient plans add their
    zeroing steps and scalar adjoints, which that count leaves out).  batch
    is the plan's B (a
    step's output holds 2^rank x B elements).  Returns {"rank>=t": bytes,
    "rank<t": bytes}."""
    sch = qb.qt_plan_schedule(plan)
    af = sch["acc_first"]
    n = len(sch["unit"])
    step = np.repeat(np.arange(n), np.diff(af))
    el = (sch["acc_hi"] - sch["acc_lo"]).astype(np.float64)
    per_step = np.bincount(step, weights=el, minlength=n)
    out_el = np.zeros(n)
    w = sch["acc_write"].astype(bool)
    np.maximum.at(out_el, step[w], el[w])
    wide = out_el >= float(batch) * 2.0 ** threshold
    return {f"rank>={threshold}": float(per_step[wide].sum() * elem_bytes),
            f"rank<{threshold}": float(per_step[~wide].sum() * elem_bytes)}


def trace_stats(trace, n_warps, bin_ns=200_000, busy_frac=0.9) -> dict:
    """Summary of a queue trace (``EnergyPlan.trace``: per task the claim,
    ready and done clock readings in ns).  A warp is *waiting* from claim to
    ready (its task's dependencies) and *working* from ready to done.

    Returns the span, the fractions of n_warps x span spent working, waiting
    and idle, the per-bin averages of working and waiting warps, and
    ``full_after_ns``: the end of the first bin in which at least busy_frac of
    the warps work (the start-up phase before it), and ``tail_ns``: the time
    from the last such bin's end to the end of the span."""
    tr = np.asarray(trace, dtype=np.uint64)
    claim, ready, done = (tr[:, i].astype(np.int64) for i in range(3))
    t0 = claim.min()
    claim, ready, done = claim - t0, ready - t0, done - t0
    span = int(done.max())
    nb = span // bin_ns + 1

    def occupancy(a, b):
        acc = np.zeros(nb + 1)
        ba, bb = a // bin_ns, b // bin_ns
        same = ba == bb
        np.add.at(acc, ba[same], (b - a)[same])
        d = ~same
        np.add.at(acc, ba[d], (ba[d] + 1) * bin_ns - a[d])
        np.add.at(acc, bb[d], b[d] - bb[d] * bin_ns)
        for k in np.nonzero(d & (bb - ba > 1))[0]:  # bins fully covered
            acc[ba[k] + 1:bb[k]] += bin_ns
        return acc[:nb] / bin_ns

    work = occupancy(ready, done)
    wait = occupancy(claim, ready)
    full = np.nonzero(work >= busy_frac * n_warps)[0]
    total = float(n_warps) * span
    return {"span_ns": span,
            "work_frac": float((done - ready).sum()) / total,
            "wait_frac": float((ready - claim).sum()) / total,
            "idle_frac": 1.0 - float((done - claim).sum()) / total,
            "working_warps": work, "waiting_warps": wait, "bin_ns": bin_ns,
            "full_after_ns": int((full[0] + 1) * bin_ns) if len(full) else None,
            "tail_ns": int(span - (full[-1] + 1) * bin_ns) if len(full) else None}


def compare(n_vertices, edges, p, **options) -> dict:
    """schedule_stats of the plan with dependency lists and with chained steps."""
    out = {}
    for name, chain in (("dependency lists", 0), ("chained", 1)):
        opt = qb.qt_plan_options_default()
        opt.mode = qb.QT_MODE_PERSISTENT
        for k, v in options.items():
            setattr(opt, k, v)
        opt.chain_steps = chain
        plan = qb.qt_plan_create(n_vertices, np.asarray(edges, dtype=np.int32), p, opt)
        try:
            out[name] = schedule_stats(plan)
        finally:
            qb.qt_plan_free(plan)
    return out


def main():
    from workloads import workload  # seeded inputs shared with the tests and the bench
    cases = [
        ("100-vertex p=4, 64 angle sets, complex64 (bench)", "n100_p4",
         dict(batch=64, dtype=qb.QT_C64, order_trials=100, group_rows=-1)),
        ("60-vertex p=4, gradient, 1 angle set", "n60_p4",
         dict(batch=1, dtype=qb.QT_C64, order_trials=100, gradient=1)),
        ("100-vertex p=4, gradient, 64 angle sets", "n100_p4",
         dict(batch=64, dtype=qb.QT_C64, order_trials=100, gradient=1)),
    ]
    for label, name, opts in cases:
        n, edges, p, _, _ = workload(name)
        res = compare(n, edges, p, **opts)
        print(label)
        for k, v in res.items():
            print(f"  {k:17s} units {v['units']:6d}  longest path {v['longest_path']:4d}  "
                  f"deps/unit {v['deps_per_unit']:.2f}  max deps {v['max_deps']}")


if __name__ == "__main__":
    main()
