"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (from the precision of each path): |d<Z_j Z_k>| <= 1e-10 for
complex128 and for float pairs (c64x2, about 48 significant bits), <= 1e-5
for complex64 (FP32 products, one FP32 add per bucket, FP64 edge product and
energy sum); the whole graph's energy E to 1e-9 (complex128, float pairs)
and 1e-5 (complex64).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lightcone as lc
from oracle import statevector as sv
from workloads import complete_graph, erdos_renyi_graph, random_angles, random_regular_graph, workload

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 1e-5, "c64x2": 1e-10}
TOL_E = {"c128": 1e-9, "c64": 1e-5, "c64x2": 1e-9}


@pytest.fixture(scope="module", autouse=True)
def _lib(qtlib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return qtlib


def _plan(n, edges, p, batch, dtype, mode, **kw):
    from paper_2106_15740_gb300.energy import EnergyPlan
    return EnergyPlan(n, edges, p, batch=batch, dtype=dtype, mode=mode, device="cuda:0", **kw)


def _run(plan, gamma, beta):
    g = torch.tensor(np.asarray(gamma).reshape(plan.batch, plan.p), device="cuda:0")
    b = torch.tensor(np.asarray(beta).reshape(plan.batch, plan.p), device="cuda:0")
    e, zz = plan.energy(g, b, edge_zz=True)
    plan.check()
    return e.cpu().numpy(), zz.cpu().numpy()


def _oracle_zz(n, edges, p, g, b, sel=None):
    sel = range(len(edges)) if sel is None else sel
    return np.array([lc.lightcone_zz(n, edges, p, g, b, e)[0] for e in sel])


# ------------------------------------------------------------ qt_contract --

@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_contract_single_networks(dtype):
    from paper_2106_15740_gb300.energy import contract_edge
    n, edges, p, g, b = workload("n16_p1")
    ref = sv.edge_zz(n, edges, g[0], b[0])
    for e in range(len(edges)):
        val, width = contract_edge(n, edges, p, g[0], b[0], e, dtype=dtype)
        assert abs(val.real - ref[e]) <= TOL[dtype]
        assert abs(val.imag) <= TOL[dtype]


def test_contract_p3_networks_c128():
    from paper_2106_15740_gb300.energy import contract_edge
    n, edges, p, g, b = workload("n100_p3")
    for e in (0, 17, 77, 149):
        val, width = contract_edge(n, edges, p, g[0], b[0], e)
        ref, w_ref = lc.lightcone_zz(n, edges, p, g[0], b[0], e)
        assert width == w_ref
        assert abs(val - ref) <= TOL["c128"]


# ------------------------------------------------------------ energy plans --

@pytest.mark.parametrize("mode", ["per_bucket", "persistent"])
@pytest.mark.parametrize("dtype", ["c128", "c64", "c64x2"])
def test_n16_p1_all_edges_vs_statevector(mode, dtype):
    n, edges, p, g, b = workload("n16_p1", batch=3)
    plan = _plan(n, edges, p, 3, dtype, mode)
    e, zz = _run(plan, g, b)
    for k in range(3):
        ref = sv.edge_zz(n, edges, g[k], b[k])
        np.testing.assert_allclose(zz[:, k, 0], ref, atol=TOL[dtype], rtol=0)
        np.testing.assert_allclose(zz[:, k, 1], 0, atol=TOL[dtype])
        assert abs(e[k] - 0.5 * (len(edges) - ref.sum())) <= TOL_E[dtype]


@pytest.mark.parametrize("mode", ["per_bucket", "persistent"])
@pytest.mark.parametrize("dtype", ["c128", "c64", "c64x2"])
def test_n100_p3_all_edges_vs_oracle(mode, dtype):
    n, edges, p, g, b = workload("n100_p3")
    plan = _plan(n, edges, p, 1, dtype, mode)
    e, zz = _run(plan, g, b)
    ref = _oracle_zz(n, edges, p, g[0], b[0])
    np.testing.assert_allclose(zz[:, 0, 0], ref.real, atol=TOL[dtype], rtol=0)
    np.testing.assert_allclose(zz[:, 0, 1], ref.imag, atol=TOL[dtype], rtol=0)
    assert abs(e[0] - 0.5 * np.sum(1 - ref.real)) <= TOL_E[dtype]


def test_n100_p4_batched_c64_vs_oracle():
    """The batched workload: 150 edges x 64 angle sets, one persistent launch.
    The oracle checks every edge on 2 angle sets and a seeded sample of
    16 edges on 4 more."""
    n, edges, p, g, b = workload("n100_p4", batch=64)
    plan = _plan(n, edges, p, 64, "c64", "persistent")
    e, zz = _run(plan, g, b)
    for k in (0, 63):
        ref = _oracle_zz(n, edges, p, g[k], b[k])
        np.testing.assert_allclose(zz[:, k, 0], ref.real, atol=TOL["c64"], rtol=0)
        np.testing.assert_allclose(zz[:, k, 1], ref.imag, atol=TOL["c64"], rtol=0)
    rng = np.random.default_rng(1234)
    sel = sorted(rng.choice(len(edges), 16, replace=False))
    for k in rng.choice(np.arange(1, 63), 4, replace=False):
        ref = _oracle_zz(n, edges, p, g[k], b[k], sel)
        np.testing.assert_allclose(zz[sel, k, 0], ref.real, atol=TOL["c64"], rtol=0)
    # energies are the edge sums
    np.testing.assert_allclose(e, 0.5 * np.sum(1 - zz[:, :, 0], axis=0), atol=1e-12)


def test_persistent_equals_per_bucket_bitwise():
    """Both modes evaluate every output element with the same arithmetic."""
    n, edges, p, g, b = workload("n100_p3", batch=4)
    out = []
    for mode in ("per_bucket", "persistent"):
        out.append(_run(_plan(n, edges, p, 4, "c128", mode), g, b)[1])
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("dtype", ["c128", "c64", "c64x2"])
@pytest.mark.parametrize("batch", [1, 2, 3, 32, 64])
def test_lean_and_generic_tiles_agree_with_oracle(dtype, batch):
    """Every batch shape of the persistent launch (the lean pair tile for one
    angle set, the lean row tile for row-wide shapes, the generic tile
    otherwise) with searched orders, against the oracle."""
    n, edges, p, g, b = workload("n100_p3", batch=batch)
    plan = _plan(n, edges, p, batch, dtype, "persistent", order_trials=4)
    _, zz = _run(plan, g, b)
    plan.close()
    sel = [0, 75, 149]
    ref = _oracle_zz(n, edges, p, g[batch - 1], b[batch - 1], sel)
    np.testing.assert_allclose(zz[sel, batch - 1, 0], ref.real, atol=TOL[dtype], rtol=0)


@pytest.mark.parametrize("batch", [2, 3, 5, 8])
def test_batch_shapes(batch):
    """Even batches use the 2-wide complex64 vectors, odd ones the scalar path."""
    n, edges = 12, random_regular_graph(12, 3, 9)
    p = 2
    g, b = random_angles(batch, p, 99)
    for dtype in ("c128", "c64"):
        plan = _plan(n, edges, p, batch, dtype, "persistent")
        e, zz = _run(plan, g, b)
        for k in range(batch):
            ref = sv.edge_zz(n, edges, g[k], b[k])
            np.testing.assert_allclose(zz[:, k, 0], ref, atol=TOL[dtype], rtol=0)


def test_edge_cases_small_graphs():
    cases = [
        (2, np.array([[0, 1]], dtype=np.int32), 1),
        (2, np.array([[0, 1]], dtype=np.int32), 3),
        (4, complete_graph(4), 2),
        (9, erdos_renyi_graph(9, 0.4, 5), 2),
        (6, np.array([[0, 1], [1, 2], [4, 5]], dtype=np.int32), 2),   # isolated vertex 3
    ]
    for n, edges, p in cases:
        g, b = random_angles(2, p, n * 10 + p)
        for dtype in ("c128", "c64"):
            for mode in ("per_bucket", "persistent"):
                plan = _plan(n, edges, p, 2, dtype, mode)
                e, zz = _run(plan, g, b)
                for k in range(2):
                    ref = sv.edge_zz(n, edges, g[k], b[k])
                    np.testing.assert_allclose(zz[:, k, 0], ref, atol=TOL[dtype], rtol=0)


def test_gamma_zero_and_symmetries_on_device():
    n, edges, p, g, b = workload("n100_p3", batch=4)
    g = g.copy()
    g[1] = 0.0                        # gamma = 0 -> E = |E|/2
    g[2], b[2] = -g[3], -b[3]         # E(-g, -b) = E(g, b)
    plan = _plan(n, edges, p, 4, "c128", "persistent")
    e, zz = _run(plan, g, b)
    assert abs(e[1] - len(edges) / 2) < 1e-10
    assert abs(e[2] - e[3]) < 1e-10
    assert np.all(np.abs(zz[:, :, 0]) <= 1 + 1e-12)


def test_host_pointer_call_matches_device_call():
    n, edges, p, g, b = workload("n100_p3", batch=2)
    plan = _plan(n, edges, p, 2, "c64", "persistent")
    e_dev, zz_dev = _run(plan, g, b)
    e_host, zz_host = plan.energy_host(g, b, edge_zz=True)
    assert np.array_equal(e_dev, e_host) and np.array_equal(zz_dev, zz_host)


def test_one_shot_qt_energy():
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, g, b = workload("n16_p1", batch=4)
    nbytes = qb.qt_energy_workspace_size(n, edges, p, 4, qb.QT_C128, 0)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda:0")
    energy = np.empty(4)
    qb.qt_energy(n, edges, p, np.ascontiguousarray(g), np.ascontiguousarray(b), 4, qb.QT_C128,
                 torch.cuda.current_stream().cuda_stream, ws.data_ptr(), nbytes, energy)
    ref = [sv.energy(n, edges, g[k], b[k]) for k in range(4)]
    np.testing.assert_allclose(energy, ref, atol=1e-9)


def test_workspace_cap_limits_concurrency():
    """A workspace cap lowers the number of edges in flight, not the result."""
    n, edges, p, g, b = workload("n100_p3", batch=2)
    full = _plan(n, edges, p, 2, "c128", "persistent")
    capped = _plan(n, edges, p, 2, "c128", "persistent", max_workspace=full.ws_bytes // 4)
    assert capped.ws_bytes < full.ws_bytes
    assert np.array_equal(_run(full, g, b)[1], _run(capped, g, b)[1])


@pytest.mark.parametrize("dtype,batch,cap", [("c64", 64, 1), ("c64", 4, 4), ("c128", 1, 4), ("c128", 3, 1)])
def test_tree_schedule_equals_chain_bitwise(dtype, batch, cap):
    """Steps that wait only for their tree dependencies (and the readers of
    the workspace they overwrite) compute every value with the same operands
    in the same order as the chained schedule: identical bits.  A workspace
    cap (cap > 1) puts several networks on one slot.  Also checked against
    the oracle."""
    n, edges, p, g, b = workload("n100_p3", batch=batch)
    out = {}
    ws = None
    for chain in (True, False):
        plan = _plan(n, edges, p, batch, dtype, "persistent", order_trials=4, chain_steps=chain,
                     max_workspace=0 if ws is None or cap == 1 else ws // cap)
        if ws is None and cap > 1:
            ws = plan.ws_bytes
            plan.close()
            plan = _plan(n, edges, p, batch, dtype, "persistent", order_trials=4, chain_steps=chain,
                         max_workspace=ws // cap)
        for _ in range(3):  # repeated launches: a race would show as a changing bit
            out.setdefault(chain, []).append(_run(plan, g, b))
        plan.close()
    for r in out[True] + out[False]:
        assert np.array_equal(r[1], out[True][0][1])
        assert np.array_equal(r[0], out[True][0][0])
    sel = [0, 75, 149]
    ref = _oracle_zz(n, edges, p, g[batch - 1], b[batch - 1], sel)
    np.testing.assert_allclose(out[False][0][1][sel, batch - 1, 0], ref.real, atol=TOL[dtype], rtol=0)


def test_workspace_too_small_is_an_error():
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, g, b = workload("n16_p1")
    plan = _plan(n, edges, p, 1, "c128", "persistent")
    gd = torch.tensor(g, device="cuda:0")
    bd = torch.tensor(b, device="cuda:0")
    out = torch.empty(1, dtype=torch.float64, device="cuda:0")
    with pytest.raises(qb.QTError) as ei:
        qb.qt_plan_energy(plan.plan, gd.data_ptr(), bd.data_ptr(), out.data_ptr(), 0, 0,
                          plan.workspace.data_ptr(), plan.ws_bytes - 1, torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == qb.QT_ENOMEM


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_searched_orders_match_oracle_on_n100_p3(dtype):
    """Plans contracted in randomised greedy orders (not min-fill) give the
    same per-edge values: all 150 edges against the oracle."""
    from paper_2106_15740_gb300.energy import EnergyPlan
    n, edges, p, g, b = workload("n100_p3", batch=1)
    plan = EnergyPlan(n, edges, p, batch=1, dtype=dtype, mode="persistent", order_trials=30, order_seed=11,
                      device="cuda:0")
    e, zz = plan.energy(torch.tensor(g, device="cuda:0"), torch.tensor(b, device="cuda:0"), edge_zz=True)
    plan.check()
    zz = zz.cpu().numpy()[:, 0, :]
    tol = 1e-10 if dtype == "c128" else 1e-5
    for ei in range(len(edges)):
        ref = lc.lightcone_zz(n, edges, p, g[0], b[0], ei)[0]
        assert abs(zz[ei, 0] - ref.real) <= tol and abs(zz[ei, 1] - ref.imag) <= tol


def test_tree_like_lightcones_give_equal_values():
    """Edges whose radius-p neighbourhood is a tree have isomorphic lightcone
    networks, so their <Z_j Z_k> must agree (to rounding: their orders and
    variable ids differ); at p = 1 they also equal the triangle-free closed
    form sin(4b) sin(2g) cos^2(2g) of a 3-regular graph."""
    from oracle import closed_form as cf
    from oracle.lightcone import reverse_lightcone
    for p, B in ((1, 2), (2, 2)):
        n = 100
        edges = random_regular_graph(n, 3, 17)
        g, b = random_angles(B, p, 18)
        tree = 2 * (2 ** (p + 1) - 1)
        like = [e for e in range(len(edges)) if len(reverse_lightcone(n, edges, p, e)[0]) == tree]
        assert len(like) >= 10
        plan = _plan(n, edges, p, B, "c128", "persistent")
        _, zz = _run(plan, g, b)
        plan.close()
        for k in range(B):
            vals = zz[like, k, 0]
            assert vals.max() - vals.min() <= 1e-12
            if p == 1:
                assert abs(vals[0] - cf.p1_zz(n, edges, like[0], g[k][0], b[k][0])) <= 1e-12


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8])
def test_tiny_graph_sweep_against_state_vector(n):
    """Every small random graph shape (G(n, 1/2), seeded) at p = 1..3, both
    precisions, both modes."""
    for seed in (1, 2):
        edges = erdos_renyi_graph(n, 0.5, 100 * n + seed)
        if len(edges) == 0:
            continue
        for p in (1, 2, 3):
            g, b = random_angles(2, p, 7 * n + p + seed)
            refs = [sv.edge_zz(n, edges, g[k], b[k]) for k in range(2)]
            for dtype in ("c128", "c64"):
                for mode in ("per_bucket", "persistent"):
                    plan = _plan(n, edges, p, 2, dtype, mode)
                    _, zz = _run(plan, g, b)
                    plan.close()
                    for k in range(2):
                        np.testing.assert_allclose(zz[:, k, 0], refs[k], atol=TOL[dtype], rtol=0)


@pytest.mark.parametrize("dtype,batch", [("c64", 64), ("c128", 1), ("c64", 1)])
def test_queue_orders_are_bitwise_identical(dtype, batch):
    """Taking the tasks with the longest remaining dependency path first, or
    in the order a list-scheduling simulation starts them, changes only when
    each step runs, not what it computes."""
    n, edges, p, g, b = workload("n100_p3", batch=batch)
    out = {}
    for order in ("round_robin", "critical_path", "simulated"):
        plan = _plan(n, edges, p, batch, dtype, "persistent", order_trials=4, queue_order=order)
        out[order] = _run(plan, g, b)
        plan.close()
    for order in ("critical_path", "simulated"):
        assert np.array_equal(out["round_robin"][1], out[order][1])
        assert np.array_equal(out["round_robin"][0], out[order][0])


def test_per_width_chunks_are_bitwise_identical():
    """Per-width schedules (warp tiles per queue task by output rank, as the
    autotuner sets them) change which warp runs which rows, not the
    arithmetic: every edge value is identical."""
    n, edges, p, g, b = workload("n100_p3", batch=64)
    out = []
    for by_rank in (None, {r: 4 for r in range(10, 32)}, {r: 2 for r in range(32)}):
        plan = _plan(n, edges, p, 64, "c64", "persistent", chunk_tiles_by_rank=by_rank)
        out.append(_run(plan, g, b))
        plan.close()
    for e, zz in out[1:]:
        assert np.array_equal(zz, out[0][1]) and np.array_equal(e, out[0][0])


def test_float_pairs_match_complex128_on_the_bench_workload():
    """The float-pair precision on the bench workload (150 edges x 64 angle
    sets, searched orders): every edge and energy against the complex128 plan
    of the same orders, to 1e-10 per edge and 1e-9 per energy."""
    n, edges, p, g, b = workload("n100_p4", batch=64)
    out = {}
    for dtype in ("c64x2", "c128"):
        plan = _plan(n, edges, p, 64, dtype, "persistent", order_trials=100)
        out[dtype] = _run(plan, g, b)
        plan.close()
    np.testing.assert_allclose(out["c64x2"][1], out["c128"][1], atol=1e-10, rtol=0)
    np.testing.assert_allclose(out["c64x2"][0], out["c128"][0], atol=1e-9, rtol=0)
