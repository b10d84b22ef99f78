"""Dependency statistics of a persistent plan's queue (host only, no device).

A persistent plan queues every step of every network in one launch; a step
waits for the steps on its dependency list (``qt_plan_schedule``).  This
module measures that graph: the number of queued units (a step's chunks, or
a group of tiny steps that one warp runs in order), the dependencies per
unit, and the longest dependency path in units, which bounds how many steps
one after another the launch must wait through.  With ``chain_steps`` every
step of a workspace slot waits for the one before it, so the path is the
length of a slot's step list.

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
