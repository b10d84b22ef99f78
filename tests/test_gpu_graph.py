"""CUDA-graph replay of a plan evaluation against direct calls and the oracle.

The batched energy step (angle table, leaf factors, one persistent launch,
FP64 energy sum) is captured once and replayed with new angles.  A replay
runs the same kernels on the same workspace as a direct call, so forward
results must agree bit for bit; gradients (atomic accumulation in the
reverse sweep) agree to rounding.  The replayed values are also checked
against the CPU oracle, complex64 within 1e-5 (the complex64 tolerance of
the other parity tests).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gradients as gr
from oracle import lightcone as lc
from workloads import random_angles, random_regular_graph, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(qtlib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return qtlib


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda:0")


@pytest.mark.parametrize("mode", ["persistent", "per_bucket"])
def test_replay_equals_direct_call_and_oracle(mode):
    from paper_2106_15740_gb300.energy import EnergyPlan
    n, edges, p, _, _ = workload("n100_p3")
    B = 4
    plan = EnergyPlan(n, edges, p, batch=B, dtype="c64", mode=mode, device="cuda:0", order_trials=8)
    cap = plan.capture(edge_zz=True)
    sel = [0, 37, 149]
    for seed in (11, 12):  # two angle sets in a row through the same graph
        g, b = random_angles(B, p, seed)
        e_rep, zz_rep = (t.clone() for t in cap(_dev(g), _dev(b)))
        e_dir, zz_dir = plan.energy(_dev(g), _dev(b), edge_zz=True)
        plan.check()
        assert torch.equal(e_rep, e_dir)
        assert torch.equal(zz_rep, zz_dir)
        zz = zz_rep.cpu().numpy()
        for k in (0, B - 1):
            ref = np.array([lc.lightcone_zz(n, edges, p, g[k], b[k], e)[0].real for e in sel])
            assert np.abs(zz[sel, k, 0] - ref).max() <= 1e-5
    plan.close()


def test_replayed_gradient_matches_direct_call_and_parameter_shift():
    from paper_2106_15740_gb300.energy import EnergyPlan
    n, p, B = 12, 2, 3
    edges = random_regular_graph(n, 3, 5)
    plan = EnergyPlan(n, edges, p, batch=B, dtype="c128", mode="persistent", gradient=True, device="cuda:0")
    cap = plan.capture(grad=True)
    for seed in (21, 22):
        g, b = random_angles(B, p, seed)
        e_rep, g_rep = (t.clone() for t in cap(_dev(g), _dev(b)))
        e_dir, g_dir = plan.energy(_dev(g), _dev(b), grad=True)
        plan.check()
        assert torch.equal(e_rep, e_dir)
        assert torch.allclose(g_rep, g_dir, rtol=0, atol=1e-12)
        for k in range(B):
            ref = np.concatenate(gr.param_shift_gradient(n, edges, g[k], b[k]))
            assert np.abs(g_rep[k].cpu().numpy() - ref).max() <= 1e-9
    plan.close()
