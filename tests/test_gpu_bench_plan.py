"""GPU parity of the exact plan the benchmark times.

The benchmark evaluates every edge lightcone of the 100-vertex p = 4 graph
(150 edges) for 64 angle sets in complex64, with per-edge searched orders
(100 randomised greedy trials), the tile its autotuner picked on the GB300
(64 items per lane, no grouping of small steps), chained buckets fused into
one step, one persistent launch replayed from a CUDA graph.  Here that plan, in that launch form, is
checked against the FP64 oracle (the lightcone contraction of
oracle/lightcone.py) on every edge for two of the 64 angle sets:

* per edge |<ZZ>_gpu - <ZZ>_oracle| <= 1e-5 (complex64 tolerance) and
  |Im <ZZ>| <= 1e-5;
* full graph |E_gpu - E_oracle| <= 1e-5, E = sum_e (1 - <ZZ>_e) / 2 over the
  150 edges (the complex64 energy tolerance).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import workload

pytestmark = pytest.mark.gpu

TOL_ZZ = 1e-5
TOL_E = 1e-5
ANGLE_SETS = (0, 63)


@pytest.fixture(scope="module")
def bench_plan_run(qtlib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_15740_gb300.energy import EnergyPlan
    n, edges, p, g, b = workload("n100_p4", batch=64)
    plan = EnergyPlan(n, edges, p, batch=64, dtype="c64", mode="persistent", order_trials=100, lane_items=64,
                      group_rows=-1, device="cuda:0")
    step = plan.capture(edge_zz=True)
    e, zz = step(torch.tensor(g, device="cuda:0"), torch.tensor(b, device="cuda:0"))
    torch.cuda.synchronize()
    plan.check()
    res = dict(n=n, edges=edges, p=p, g=g, b=b, energy=e.cpu().numpy().copy(), zz=zz.cpu().numpy().copy(),
               widths=plan.widths.copy(), alg=plan.stats["alg_bytes"])
    plan.close()
    return res


@pytest.fixture(scope="module")
def oracle_zz(bench_plan_run):
    import multiprocessing as mp
    import os
    import oracle_workers
    oracle_workers.single_threaded()
    jobs = [("n100_p4", 64, e, k) for k in ANGLE_SETS for e in range(len(bench_plan_run["edges"]))]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        vals = pool.map(oracle_workers.lightcone_zz, jobs, chunksize=4)
    return {(e, k): v for (_, _, e, k), v in zip(jobs, vals)}


def test_bench_plan_is_the_timed_plan(bench_plan_run):
    """Searched orders: widths 10..20; 36.2 GB stored and read per evaluation
    by the chained steps, 82.7 GB with every bucket a step of its own (the
    bucket-by-bucket figure the benchmark's roofline divides)."""
    from paper_2106_15740_gb300 import binding as qb
    r = bench_plan_run
    assert r["widths"].min() >= 10 and r["widths"].max() <= 20
    assert abs(r["alg"] - 36202615808.0) / 36202615808.0 < 1e-9
    opt = qb.qt_plan_options_default()
    opt.batch, opt.dtype, opt.mode, opt.order_trials = 64, qb.QT_C64, qb.QT_MODE_PERSISTENT, 100
    opt.lane_items, opt.group_rows, opt.fuse_chains = 64, -1, 0
    plan = qb.qt_plan_create(r["n"], r["edges"], r["p"], opt)
    try:
        assert abs(qb.qt_plan_stats(plan)["alg_bytes"] - 82730662912.0) / 82730662912.0 < 1e-9
    finally:
        qb.qt_plan_free(plan)


def test_every_edge_matches_oracle(bench_plan_run, oracle_zz):
    r = bench_plan_run
    for k in ANGLE_SETS:
        for e in range(len(r["edges"])):
            ref = oracle_zz[(e, k)]
            assert abs(r["zz"][e, k, 0] - ref.real) <= TOL_ZZ, (e, k)
            assert abs(r["zz"][e, k, 1]) <= TOL_ZZ


def test_energy_matches_oracle(bench_plan_run, oracle_zz):
    r = bench_plan_run
    for k in ANGLE_SETS:
        e_ref = sum(0.5 * (1.0 - oracle_zz[(e, k)].real) for e in range(len(r["edges"])))
        assert abs(r["energy"][k] - e_ref) <= TOL_E, (k, r["energy"][k] - e_ref)
