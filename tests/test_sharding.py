"""Host-side sharding of one graph's edges between ranks: the contiguous
cost-balanced partition, the per-edge cost model, and the single sum
reduction, the latter on two gloo ranks on the CPU."""
import itertools
import json
import socket
import subprocess
import sys
from pathlib import Path

import numpy as np
import pytest

from oracle import statevector as sv
from workloads import random_angles, random_regular_graph, workload

ROOT = Path(__file__).resolve().parent.parent


def _best_max_by_brute_force(costs, world):
    m = len(costs)
    best = np.inf
    for cuts in itertools.combinations(range(1, m), min(world, m) - 1):
        bounds = (0,) + cuts + (m,)
        best = min(best, max(sum(costs[bounds[i]:bounds[i + 1]]) for i in range(len(bounds) - 1)))
    return best


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_partition_is_an_optimal_contiguous_split(seed, world):
    from paper_2106_15740_gb300.sharding import partition
    rng = np.random.default_rng(seed)
    costs = rng.integers(1, 100, size=int(rng.integers(1, 10))).astype(float)
    ranges = partition(costs, world)
    assert len(ranges) == world
    assert ranges[0][0] == 0 and ranges[-1][1] == len(costs)
    for (a0, b0), (a1, b1) in zip(ranges, ranges[1:]):
        assert b0 == a1 and a0 <= b0
    nonempty = [r for r in ranges if r[1] > r[0]]
    assert len(nonempty) == min(world, len(costs))
    worst = max(costs[a:b].sum() for a, b in ranges)
    assert worst <= _best_max_by_brute_force(list(costs), world) * (1 + 1e-9)


def test_edge_costs_split_the_plan_total(qtlib):
    from paper_2106_15740_gb300 import binding as qb
    from paper_2106_15740_gb300.sharding import edge_costs
    n, edges, p, g, b = workload("n100_p3")
    c = edge_costs(n, edges, p, batch=4)
    opt = qb.qt_plan_options_default()
    opt.batch = 4
    opt.dtype = qb.QT_C64
    plan = qb.qt_plan_create(n, edges, p, opt)
    total = qb.qt_plan_stats(plan)["alg_bytes"]
    qb.qt_plan_free(plan)
    assert len(c) == len(edges) and (c > 0).all()
    assert abs(c.sum() - total) <= 1e-9 * total
    # a sub-range plan gives the same per-edge costs
    opt.edge_begin, opt.edge_end = 10, 30
    plan = qb.qt_plan_create(n, edges, p, opt)
    sub = qb.qt_plan_edge_bytes(plan, 20)
    qb.qt_plan_free(plan)
    np.testing.assert_array_equal(sub, c[10:30])
    # slicing multiplies an edge's networks: its cost goes up, the others stay
    cs = edge_costs(n, edges, p, batch=4, max_width=9, slice=True)
    widths = np.array([w for w in _widths(n, edges, p)])
    np.testing.assert_array_equal(cs[widths <= 9], c[widths <= 9])


def _widths(n, edges, p):
    from paper_2106_15740_gb300 import binding as qb
    opt = qb.qt_plan_options_default()
    plan = qb.qt_plan_create(n, edges, p, opt)
    w = qb.qt_plan_edge_widths(plan, len(edges))
    qb.qt_plan_free(plan)
    return w


def test_two_gloo_ranks_sum_their_edge_ranges(qtlib, tmp_path):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           str(ROOT / "tests" / "gloo_shard_worker.py"), str(tmp_path)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    res = [json.loads((tmp_path / f"rank{k}.json").read_text()) for k in range(2)]
    n, p, B = 12, 2, 2
    edges = random_regular_graph(n, 3, 21)
    g, b = random_angles(B, p, 77)
    ranges = res[0]["ranges"]
    assert ranges == res[1]["ranges"] and ranges[0][0] == 0 and ranges[0][1] == ranges[1][0]
    assert ranges[1][1] == len(edges) and ranges[0][1] > 0 and ranges[1][1] > ranges[1][0]
    for k in range(B):
        exact = sv.energy(n, edges, g[k], b[k])
        for r in res:
            assert abs(r["energy"][k] - exact) < 1e-10
        assert abs(res[0]["partial"][k] + res[1]["partial"][k] - exact) < 1e-10
    for r in res:
        np.testing.assert_array_equal(np.array(r["grad"]), np.full((B, 2 * p), 3.0))
