"""GPU parity of sliced edge networks.

Slicing fixes s variables of an edge's network and sums the 2^s restricted
networks; the sum is the unsliced value exactly (a sum over a variable split
into its two terms), so every comparison is with the oracle's unsliced
result: the 2^n state vector for small graphs, the oracle's lightcone
contraction for sampled edges of the 100-vertex graphs, and the parameter-shift
gradient for the adjoint sweep over sliced networks.

Tolerances: complex128 1e-10 per edge <ZZ> (a few thousand FP64 products and
sums per network, at most 2^10 networks); complex64 1e-5 per edge <ZZ>.
Energies are compared with their own tolerance: 1e-9 (complex128) and 1e-5
(complex64) for the whole graph's E, not the per-edge one scaled by the
edge count.
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


def _plan(n, edges, p, B, dtype, mode, max_width, **kw):
    from paper_2106_15740_gb300.energy import EnergyPlan
    return EnergyPlan(n, edges, p, batch=B, dtype=dtype, mode=mode, max_width=max_width, slice=True,
                      device="cuda:0", **kw)


def _dev(x, plan):
    return torch.tensor(np.asarray(x).reshape(plan.batch, plan.p), device="cuda:0")


@pytest.mark.parametrize("mode", ["per_bucket", "persistent"])
@pytest.mark.parametrize("dtype", ["c128", "c64", "c64x2"])
@pytest.mark.parametrize("n,p,B,max_width,seed", [(16, 1, 2, 2, 0), (12, 2, 3, 3, 5), (14, 3, 2, 4, 6)])
def test_sliced_energy_matches_state_vector(mode, dtype, n, p, B, max_width, seed):
    edges = random_regular_graph(n, 3, seed)
    g, b = random_angles(B, p, 90 + seed)
    plan = _plan(n, edges, p, B, dtype, mode, max_width)
    assert plan.slices.max() > 0 and plan.widths.max() <= max_width
    e = plan.energy(_dev(g, plan), _dev(b, plan)).cpu().numpy()
    plan.check()
    tol = 1e-5 if dtype == "c64" else 1e-9
    for k in range(B):
        assert abs(e[k] - sv.energy(n, edges, g[k], b[k])) <= tol


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_sliced_n100_p3_edges_match_oracle(dtype):
    """Budget 9 on the 100-vertex p = 3 graph (widths 7..14): the per-edge
    <ZZ> of sliced and unsliced edges against the oracle's contraction."""
    n, edges, p, g, b = workload("n100_p3", batch=2)
    plan = _plan(n, edges, p, 2, dtype, "persistent", 9)
    assert (plan.slices > 0).sum() >= 20
    e, zz = plan.energy(_dev(g, plan), _dev(b, plan), edge_zz=True)
    plan.check()
    zz = zz.cpu().numpy()
    tol = 1e-10 if dtype == "c128" else 1e-5
    sample = sorted(set(np.flatnonzero(plan.slices > 0)[:12]) | {0, 75, 149})
    for k in range(2):
        for ei in sample:
            ref = lc.lightcone_zz(n, edges, p, g[k], b[k], int(ei))[0]
            assert abs(zz[ei, k, 0] - ref.real) <= tol and abs(zz[ei, k, 1] - ref.imag) <= tol


def test_sliced_plan_equals_unsliced_plan_on_n60_p4():
    """The 60-vertex p = 4 graph at budget 21 (widths up to 27): every edge's
    <ZZ> from the sliced plan against the unsliced complex128 plan."""
    from paper_2106_15740_gb300.energy import EnergyPlan
    n, edges, p, g, b = workload("n60_p4", batch=2)
    full = EnergyPlan(n, edges, p, batch=2, dtype="c128", mode="persistent", device="cuda:0")
    sl = _plan(n, edges, p, 2, "c128", "persistent", 21)
    assert sl.slices.max() >= 3
    _, z0 = full.energy(_dev(g, full), _dev(b, full), edge_zz=True)
    _, z1 = sl.energy(_dev(g, sl), _dev(b, sl), edge_zz=True)
    sl.check()
    np.testing.assert_allclose(z1.cpu().numpy(), z0.cpu().numpy(), atol=1e-10, rtol=0)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,p,B,max_width,seed", [(12, 2, 2, 3, 5), (10, 3, 2, 4, 7)])
def test_sliced_gradient_matches_parameter_shift(dtype, n, p, B, max_width, seed):
    edges = random_regular_graph(n, 3, seed)
    g, b = random_angles(B, p, 70 + seed)
    plan = _plan(n, edges, p, B, dtype, "persistent", max_width, gradient=True)
    assert plan.slices.max() > 0
    e, grad = plan.energy(_dev(g, plan), _dev(b, plan), grad=True)
    plan.check()
    grad = grad.cpu().numpy()
    for k in range(B):
        ref = np.concatenate(gr.param_shift_gradient(n, edges, g[k], b[k]))
        tol = 1e-9 if dtype == "c128" else 5e-5 * max(1.0, np.abs(ref).max())
        np.testing.assert_allclose(grad[k], ref, atol=tol, rtol=0)



@pytest.mark.parametrize("n,p,max_width,seed", [(12, 2, 3, 5), (10, 3, 4, 7)])
def test_sliced_float_pair_gradient_matches_parameter_shift(n, p, max_width, seed):
    """Float-pair gradients (one angle set) on sliced networks: the slices'
    leaf-factor adjoints are summed in FP64; complex128 tolerance."""
    edges = random_regular_graph(n, 3, seed)
    g, b = random_angles(1, p, 70 + seed)
    plan = _plan(n, edges, p, 1, "c64x2", "persistent", max_width, gradient=True)
    assert plan.slices.max() > 0
    e, grad = plan.energy(_dev(g, plan), _dev(b, plan), grad=True)
    plan.check()
    ref = np.concatenate(gr.param_shift_gradient(n, edges, g[0], b[0]))
    np.testing.assert_allclose(grad.cpu().numpy()[0], ref, atol=1e-9, rtol=0)