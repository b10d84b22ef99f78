"""GPU parity of the adjoint gradient dE/dgamma, dE/dbeta (reverse bucket sweep).

References: the oracle's parameter-shift gradient on a 2^n state vector
(exact), central finite differences (h = 1e-5) of the oracle's lightcone
energy for a seeded sample of single edges, and central finite differences
of the complex128 GPU energy for the whole 60-vertex p = 4 graph.

Tolerances: complex128 1e-9 absolute against the exact gradient (rounding of
a few thousand FP64 products and sums); against finite differences the FD
truncation error O(h^2 |E'''|) ~ 1e-8 dominates.  complex64: 1e-5 per unit of
gradient scale (FP32 rounding, about 100 bucket steps of 2^-24 each; the
stored gates' norm is divided out per network).  Energies: 1e-9 (complex128)
and 1e-5 (complex64) for the whole graph.  Float pairs (one angle set) take
the complex128 tolerances.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gradients as gr
from oracle import lightcone as lc
from oracle import statevector as sv
from workloads import random_angles, random_regular_graph, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(qtlib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return qtlib


def _grad_plan(n, edges, p, B, dtype, **kw):
    from paper_2106_15740_gb300.energy import EnergyPlan
    return EnergyPlan(n, edges, p, batch=B, dtype=dtype, mode="persistent", gradient=True, device="cuda:0", **kw)


def _run(plan, g, b):
    gd = torch.tensor(np.asarray(g).reshape(plan.batch, plan.p), device="cuda:0")
    bd = torch.tensor(np.asarray(b).reshape(plan.batch, plan.p), device="cuda:0")
    e, grad = plan.energy(gd, bd, grad=True)
    plan.check()
    return e.cpu().numpy(), grad.cpu().numpy()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,p,B,seed", [(12, 2, 2, 5), (14, 3, 1, 6), (10, 3, 3, 7)])
def test_gradient_matches_parameter_shift(dtype, n, p, B, seed):
    edges = random_regular_graph(n, 3, seed)
    g, b = random_angles(B, p, 70 + seed)
    plan = _grad_plan(n, edges, p, B, dtype)
    e, grad = _run(plan, g, b)
    for k in range(B):
        dg, db = gr.param_shift_gradient(n, edges, g[k], b[k])
        ref = np.concatenate([dg, db])
        scale = max(1.0, np.abs(ref).max())
        tol = 1e-9 if dtype == "c128" else 1e-5 * scale
        np.testing.assert_allclose(grad[k], ref, atol=tol, rtol=0)
        assert abs(e[k] - sv.energy(n, edges, g[k], b[k])) <= (1e-9 if dtype == "c128" else 1e-5)


@pytest.mark.parametrize("n,p,B,seed", [(14, 3, 1, 6), (12, 2, 1, 5), (16, 3, 1, 8), (12, 2, 2, 5), (10, 3, 3, 7),
                                        (12, 2, 5, 9)])
def test_float_pair_gradient_matches_parameter_shift(n, p, B, seed):
    """Float pairs (one angle set on the pair tiles, 2 to 16 on the
    multi-row tiles): complex128-class, so the complex128 tolerances (1e-9
    against the exact gradient and energy)."""
    edges = random_regular_graph(n, 3, seed)
    g, b = random_angles(B, p, 70 + seed)
    e, grad = _run(_grad_plan(n, edges, p, B, "c64x2"), g, b)
    for k in range(B):
        dg, db = gr.param_shift_gradient(n, edges, g[k], b[k])
        np.testing.assert_allclose(grad[k], np.concatenate([dg, db]), atol=1e-9, rtol=0)
        assert abs(e[k] - sv.energy(n, edges, g[k], b[k])) <= 1e-9


@pytest.mark.parametrize("trials", [0, 100])
def test_n60_p4_float_pair_gradient_equals_complex128(trials):
    """Whole 60-vertex p = 4 graph (every adjoint tile shape of one angle set,
    the reduction steps with lanes on completions and on the low variables,
    atomic adds from many warps per target): float pairs against complex128
    at 1e-10 per unit of gradient scale (both sum the same terms; float pairs
    carry about 48 significant bits, and the complex128 gradient is pinned to
    the oracle's finite differences above)."""
    n, edges, p, g, b = workload("n60_p4")
    e2, grad2 = _run(_grad_plan(n, edges, p, 1, "c64x2", order_trials=trials), g, b)
    e1, grad1 = _run(_grad_plan(n, edges, p, 1, "c128", order_trials=trials), g, b)
    scale = max(1.0, np.abs(grad1).max())
    np.testing.assert_allclose(grad2, grad1, atol=1e-10 * scale, rtol=0)
    np.testing.assert_allclose(e2, e1, atol=1e-10, rtol=0)


def test_gradient_plan_energy_equals_forward_plan():
    """The forward part of a gradient plan keeps every intermediate; the
    energies must be the ones the forward-only plan gives."""
    from paper_2106_15740_gb300.energy import EnergyPlan
    n, edges, p, g, b = workload("n100_p3", batch=2)
    fwd = EnergyPlan(n, edges, p, batch=2, dtype="c128", mode="persistent", device="cuda:0")
    gd, bd = torch.tensor(g, device="cuda:0"), torch.tensor(b, device="cuda:0")
    e_fwd = fwd.energy(gd, bd).cpu().numpy()
    e_grad, _ = _run(_grad_plan(n, edges, p, 2, "c128"), g, b)
    np.testing.assert_allclose(e_grad, e_fwd, atol=1e-12, rtol=0)


def test_n60_p4_single_edges_vs_oracle_finite_differences():
    """Edge-range plans give dZ_e-based gradients of one edge's energy term;
    compare with central differences of the oracle's lightcone value."""
    n, edges, p, g, b = workload("n60_p4")
    rng = np.random.default_rng(4)
    h = 1e-5
    for e in sorted(rng.choice(len(edges), 4, replace=False)):
        plan = _grad_plan(n, edges, p, 1, "c128", edge_range=(int(e), int(e) + 1))
        energy, grad = _run(plan, g, b)

        def e_term(gg, bb):
            return 0.5 * (1.0 - lc.lightcone_zz(n, edges, p, gg, bb, int(e))[0].real)

        dg, db = gr.fd_gradient(e_term, g[0], b[0], h=h)
        np.testing.assert_allclose(grad[0], np.concatenate([dg, db]), atol=2e-8, rtol=0)
        assert abs(energy[0] - e_term(g[0], b[0])) < 1e-10


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_n60_p4_full_graph_vs_gpu_finite_differences(dtype):
    """Whole 90-edge graph: the adjoint gradient against central differences
    of the complex128 GPU energy (forward plan, h = 1e-5)."""
    from paper_2106_15740_gb300.energy import EnergyPlan
    n, edges, p, g, b = workload("n60_p4")
    e, grad = _run(_grad_plan(n, edges, p, 1, dtype), g, b)
    fwd = EnergyPlan(n, edges, p, batch=1, dtype="c128", mode="persistent", device="cuda:0")
    h = 1e-5

    def energy(gg, bb):
        return float(fwd.energy(torch.tensor(gg.reshape(1, p), device="cuda:0"),
                                torch.tensor(bb.reshape(1, p), device="cuda:0")).cpu().numpy()[0])

    dg, db = gr.fd_gradient(energy, g[0], b[0], h=h)
    ref = np.concatenate([dg, db])
    tol = 1e-7 if dtype == "c128" else 1e-5 * max(1.0, np.abs(ref).max())
    np.testing.assert_allclose(grad[0], ref, atol=tol, rtol=0)


def test_gradient_requires_gradient_plan():
    from paper_2106_15740_gb300 import binding as qb
    from paper_2106_15740_gb300.energy import EnergyPlan
    n, edges, p, g, b = workload("n16_p1")
    plan = EnergyPlan(n, edges, p, batch=1, dtype="c128", mode="persistent", device="cuda:0")
    with pytest.raises(qb.QTError) as ei:
        plan.energy(torch.tensor(g, device="cuda:0"), torch.tensor(b, device="cuda:0"), grad=True)
    assert ei.value.status == qb.QT_ESTATE


def test_autograd_function_matches_parameter_shift():
    """QAOAEnergy through torch.autograd: the gradient of sum_k w_k E_k is
    w_k times the parameter-shift gradient of angle set k."""
    from paper_2106_15740_gb300.energy import qaoa_energy
    n, p, B = 12, 2, 3
    edges = random_regular_graph(n, 3, 11)
    g, b = random_angles(B, p, 123)
    plan = _grad_plan(n, edges, p, B, "c128")
    gd = torch.tensor(g, device="cuda:0", requires_grad=True)
    bd = torch.tensor(b, device="cuda:0", requires_grad=True)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda:0")
    e = qaoa_energy(plan, gd, bd)
    (e * w).sum().backward()
    plan.check()
    for k in range(B):
        dg, db = gr.param_shift_gradient(n, edges, g[k], b[k])
        np.testing.assert_allclose(gd.grad[k].cpu().numpy(), w[k].item() * dg, atol=1e-9, rtol=0)
        np.testing.assert_allclose(bd.grad[k].cpu().numpy(), w[k].item() * db, atol=1e-9, rtol=0)
        assert abs(e[k].item() - sv.energy(n, edges, g[k], b[k])) < 1e-9


def test_autograd_function_without_gradient_plan():
    """A forward-only plan serves angle tensors that need no gradient and
    refuses those that do."""
    from paper_2106_15740_gb300 import binding as qb
    from paper_2106_15740_gb300.energy import EnergyPlan, qaoa_energy
    n, edges, p, g, b = workload("n16_p1")
    plan = EnergyPlan(n, edges, p, batch=1, dtype="c128", mode="persistent", device="cuda:0")
    e = qaoa_energy(plan, torch.tensor(g, device="cuda:0"), torch.tensor(b, device="cuda:0"))
    assert abs(e.item() - sv.energy(n, edges, g[0], b[0])) < 1e-9
    with pytest.raises(qb.QTError) as ei:
        qaoa_energy(plan, torch.tensor(g, device="cuda:0", requires_grad=True), torch.tensor(b, device="cuda:0"))
    assert ei.value.status == qb.QT_ESTATE


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_gradient_with_searched_orders_matches_parameter_shift(dtype):
    n, p, B = 14, 3, 2
    edges = random_regular_graph(n, 3, 6)
    g, b = random_angles(B, p, 76)
    plan = _grad_plan(n, edges, p, B, dtype, order_trials=20, order_seed=5)
    e, grad = _run(plan, g, b)
    for k in range(B):
        ref = np.concatenate(gr.param_shift_gradient(n, edges, g[k], b[k]))
        tol = 1e-9 if dtype == "c128" else 1e-5 * max(1.0, np.abs(ref).max())
        np.testing.assert_allclose(grad[k], ref, atol=tol, rtol=0)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("budget", [1 << 9, 1 << 12, 1 << 16])
def test_checkpointed_gradient_matches_full_sweep_and_parameter_shift(dtype, budget):
    """Checkpoint segments (forward steps re-run in the reverse sweep) give
    the same E and gradient as keeping every intermediate, up to rounding
    order, and match the exact parameter-shift gradient."""
    n, p, B = 14, 3, 2
    edges = random_regular_graph(n, 3, 11)
    g, b = random_angles(B, p, 91)
    full = _grad_plan(n, edges, p, B, dtype)
    e0, g0 = _run(full, g, b)
    full.close()
    plan = _grad_plan(n, edges, p, B, dtype, checkpoint_bytes=budget)
    assert plan.stats["alg_bytes"] > 0
    e1, g1 = _run(plan, g, b)
    plan.close()
    tol = 1e-12 if dtype == "c128" else 1e-5
    np.testing.assert_allclose(e1, e0, atol=1e-10 if dtype == "c128" else 1e-5, rtol=0)
    np.testing.assert_allclose(g1, g0, atol=tol * max(1.0, np.abs(g0).max()), rtol=0)
    for k in range(B):
        ref = np.concatenate(gr.param_shift_gradient(n, edges, g[k], b[k]))
        np.testing.assert_allclose(g1[k], ref, atol=1e-9 if dtype == "c128" else 1e-5 * max(1.0, np.abs(ref).max()),
                                   rtol=0)


@pytest.mark.parametrize("B", [4, 16])
def test_n60_p4_batched_float_pair_gradient_equals_complex128(B):
    """The multi-row float-pair gradient (4 and 16 angle sets: 8 and 2 rows
    per warp pass) on the whole 60-vertex p = 4 graph against complex128 at
    1e-10 per unit of gradient scale.  Searched orders (100 trials per edge):
    at 16 angle sets a min-fill plan would need 658 GiB of workspace, the
    searched one 81 GiB."""
    n, edges, p, _, _ = workload("n60_p4")
    g, b = random_angles(B, p, 1003)
    e2, grad2 = _run(_grad_plan(n, edges, p, B, "c64x2", order_trials=100), g, b)
    e1, grad1 = _run(_grad_plan(n, edges, p, B, "c128", order_trials=100), g, b)
    scale = max(1.0, np.abs(grad1).max())
    np.testing.assert_allclose(grad2, grad1, atol=1e-10 * scale, rtol=0)
    np.testing.assert_allclose(e2, e1, atol=1e-10, rtol=0)


@pytest.mark.parametrize("budget", [1 << 9, 1 << 12])
def test_float_pair_checkpointed_gradient(budget):
    """Float pairs (one angle set) with checkpoint segments: forward steps
    re-run in the reverse sweep read float pairs, adjoints stay FP64; the
    same gradient as the full sweep and the exact one at complex128
    tolerances."""
    n, p = 14, 3
    edges = random_regular_graph(n, 3, 11)
    g, b = random_angles(1, p, 91)
    e0, g0 = _run(_grad_plan(n, edges, p, 1, "c64x2"), g, b)
    plan = _grad_plan(n, edges, p, 1, "c64x2", checkpoint_bytes=budget)
    e1, g1 = _run(plan, g, b)
    np.testing.assert_allclose(e1, e0, atol=1e-12, rtol=0)
    np.testing.assert_allclose(g1, g0, atol=1e-12 * max(1.0, np.abs(g0).max()), rtol=0)
    ref = np.concatenate(gr.param_shift_gradient(n, edges, g[0], b[0]))
    np.testing.assert_allclose(g1[0], ref, atol=1e-9, rtol=0)


def test_checkpointed_gradient_on_n60_p4_edges():
    """A larger checkpointed plan (10 edges of the 60-vertex p = 4 graph,
    complex128) against the unsegmented sweep."""
    n, edges, p, g, b = workload("n60_p4")
    out = []
    for cb in (0, 1 << 22):
        plan = _grad_plan(n, edges, p, 1, "c128", edge_range=(0, 10), checkpoint_bytes=cb)
        out.append(_run(plan, g, b))
        plan.close()
    np.testing.assert_allclose(out[1][0], out[0][0], atol=1e-11, rtol=0)
    np.testing.assert_allclose(out[1][1], out[0][1], atol=1e-11, rtol=0)


@pytest.mark.parametrize("dtype,B,checkpoint,cap", [("c128", 1, 0, 1), ("c128", 2, 1 << 12, 2), ("c64", 64, 0, 1),
                                                    ("c64", 3, 0, 2)])
def test_tree_schedule_gradient_equals_chain(dtype, B, checkpoint, cap):
    """Adjoint steps that wait only for what they read and for the users of
    the space they reuse give the chained schedule's E and gradient: E
    bit for bit, the gradient up to the order of the atomic additions of
    accumulating adjoint steps.  cap = 2 halves the data region so that
    networks share a workspace slot.  Repeated launches check that nothing
    changes from run to run beyond that order; one angle set is checked
    against the exact parameter-shift gradient."""
    n, p = 14, 3
    edges = random_regular_graph(n, 3, 12)
    g, b = random_angles(B, p, 93)
    out = {}
    data = None
    for chain in (True, False):
        kw = dict(checkpoint_bytes=checkpoint, chain_steps=chain)
        if cap > 1:
            if data is None:
                from paper_2106_15740_gb300 import binding as qb
                probe = _grad_plan(n, edges, p, B, dtype, checkpoint_bytes=checkpoint)
                data = int(qb.qt_plan_schedule(probe.plan)["acc_hi"].max()) * (16 if dtype == "c128" else 8)
                probe.close()
            kw["max_workspace"] = data * 2 // 3
        plan = _grad_plan(n, edges, p, B, dtype, **kw)
        out[chain] = [_run(plan, g, b) for _ in range(3)]
        plan.close()
    e0, g0 = out[True][0]
    tol = 1e-12 if dtype == "c128" else 2e-6
    for e, gg in out[True] + out[False]:
        assert np.array_equal(e, e0)
        np.testing.assert_allclose(gg, g0, atol=tol * max(1.0, np.abs(g0).max()), rtol=0)
    k = B - 1
    ref = np.concatenate(gr.param_shift_gradient(n, edges, g[k], b[k]))
    np.testing.assert_allclose(out[False][0][1][k], ref,
                               atol=1e-9 if dtype == "c128" else 1e-5 * max(1.0, np.abs(ref).max()), rtol=0)


def test_n20_p2_gradient_vs_state_vector_differences():
    """A 2^20-amplitude reference: a seeded 20-vertex 3-regular graph at
    p = 2, the complex128 GPU energy and gradient against the exact
    state-vector energy and its central differences (h = 1e-5; truncation
    and rounding below 1e-8 here, checked against the parameter-shift rule,
    which takes minutes at this size and is pinned against these
    differences on smaller graphs in the oracle tests)."""
    n, p, B = 20, 2, 1
    edges = random_regular_graph(n, 3, 20)
    g, b = random_angles(B, p, 1020)
    plan = _grad_plan(n, edges, p, B, "c128")
    e, grad = _run(plan, g, b)
    plan.close()
    assert abs(e[0] - sv.energy(n, edges, g[0], b[0])) <= 1e-9
    dg, db = gr.fd_gradient(lambda gg, bb: sv.energy(n, edges, gg, bb), g[0], b[0])
    ref = np.concatenate([dg, db])
    np.testing.assert_allclose(grad[0], ref, atol=1e-7 * max(1.0, np.abs(ref).max()), rtol=0)
