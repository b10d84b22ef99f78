"""The 244-vertex p = 5 graph (366 edges, unsliced widths 14..38): every edge
above the width budget is sliced.

References: the oracle's lightcone contraction on a seeded sample of narrow
edges (width <= 18, seconds each on the CPU); for sliced edges, complex128
plans sliced at a different budget (other sliced variables, other orders);
invariants on all edges (|<ZZ>| <= 1, Im <ZZ> = 0, E = sum (1 - Re)/2).
Tolerance 2e-5 per edge for complex64 (FP32 rounding over a few hundred
bucket steps per network, networks summed in FP64).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lightcone as lc
from workloads import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sliced_run(qtlib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_15740_gb300.energy import EnergyPlan
    torch.cuda.empty_cache()
    n, edges, p, g, b = workload("n244_p5")
    plan = EnergyPlan(n, edges, p, batch=1, dtype="c64", mode="persistent", max_width=30, slice=True,
                      max_workspace=64 << 30, device="cuda:0")
    gd, bd = torch.tensor(g, device="cuda:0"), torch.tensor(b, device="cuda:0")
    e, zz = plan.energy(gd, bd, edge_zz=True)
    plan.check()
    res = dict(n=n, edges=edges, p=p, g=g, b=b, energy=e.cpu().numpy(), zz=zz.cpu().numpy(),
               widths=plan.widths.copy(), slices=plan.slices.copy())
    plan.close()
    del plan
    torch.cuda.empty_cache()
    return res


def test_widths_within_budget_and_invariants(sliced_run):
    r = sliced_run
    assert (r["widths"] <= 30).all() and (r["slices"] > 0).sum() >= 40
    zz = r["zz"][:, 0, :]
    assert np.abs(zz[:, 1]).max() < 2e-5
    assert np.abs(zz[:, 0]).max() <= 1 + 2e-5
    e_sum = 0.5 * (1.0 - zz[:, 0]).sum()
    assert abs(r["energy"][0] - e_sum) < 1e-9
    assert 0 <= r["energy"][0] <= len(r["edges"])


def test_narrow_edges_match_oracle(sliced_run):
    r = sliced_run
    narrow = np.flatnonzero((r["widths"] <= 18) & (r["slices"] == 0))
    rng = np.random.default_rng(244)
    for e in sorted(rng.choice(narrow, 6, replace=False)):
        ref = lc.lightcone_zz(r["n"], r["edges"], r["p"], r["g"][0], r["b"][0], int(e))[0]
        assert abs(r["zz"][e, 0, 0] - ref.real) < 2e-5 and abs(r["zz"][e, 0, 1] - ref.imag) < 2e-5


def test_sliced_edges_match_complex128_at_another_budget(sliced_run):
    from paper_2106_15740_gb300.energy import EnergyPlan
    r = sliced_run
    sliced = np.flatnonzero(r["slices"] > 0)
    rng = np.random.default_rng(2445)
    gd, bd = torch.tensor(r["g"], device="cuda:0"), torch.tensor(r["b"], device="cuda:0")
    for e in sorted(rng.choice(sliced, 3, replace=False)):
        plan = EnergyPlan(r["n"], r["edges"], r["p"], batch=1, dtype="c128", mode="persistent", max_width=27,
                          slice=True, edge_range=(int(e), int(e) + 1), max_workspace=48 << 30, device="cuda:0")
        assert plan.slices[0] > r["slices"][e]
        _, zz = plan.energy(gd, bd, edge_zz=True)
        plan.check()
        zz = zz.cpu().numpy()[0, 0]
        assert abs(r["zz"][e, 0, 0] - zz[0]) < 2e-5 and abs(zz[1]) < 1e-10
        plan.close()


def test_searched_order_plan_agrees_with_min_fill_plan(sliced_run):
    """With the order search the graph needs far fewer sliced edges; every
    edge's <ZZ> agrees with the min-fill sliced plan."""
    from paper_2106_15740_gb300.energy import EnergyPlan
    r = sliced_run
    plan = EnergyPlan(r["n"], r["edges"], r["p"], batch=1, dtype="c64", mode="persistent", max_width=30, slice=True,
                      order_trials=20, max_workspace=64 << 30, device="cuda:0")
    assert (plan.widths <= 30).all() and plan.slices.sum() < r["slices"].sum()
    gd, bd = torch.tensor(r["g"], device="cuda:0"), torch.tensor(r["b"], device="cuda:0")
    e, zz = plan.energy(gd, bd, edge_zz=True)
    plan.check()
    np.testing.assert_allclose(zz.cpu().numpy()[:, 0, 0], r["zz"][:, 0, 0], atol=4e-5, rtol=0)
    plan.close()
