"""The 244-vertex p = 5 graph (366 edges, unsliced widths 14..38): every edge
above the width budget is sliced.

References: the oracle's lightcone contraction on a seeded sample of narrow
edges (width <= 18, seconds each on the CPU); for sliced edges, complex128
plans sliced at a different budget (other sliced variables, other orders);
invariants on all edges (|<ZZ>| <= 1, Im <ZZ> = 0, E = sum (1 - Re)/2);
gradients of single edges against central differences.  Tolerance 1e-5 per
edge <ZZ> (and per gradient component, relative to the gradient's size) for
complex64; the two complex64 plans (different orders and slices) agree to
2e-5, the sum of two such errors.
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
    assert np.abs(zz[:, 1]).max() < 1e-5
    assert np.abs(zz[:, 0]).max() <= 1 + 1e-5
    e_sum = 0.5 * (1.0 - zz[:, 0]).sum()
    assert abs(r["energy"][0] - e_sum) < 1e-9
    assert 0 <= r["energy"][0] <= len(r["edges"])


def test_narrow_edges_match_oracle(sliced_run):
    r = sliced_run
    narrow = np.flatnonzero((r["widths"] <= 18) & (r["slices"] == 0))
    rng = np.random.default_rng(244)
    for e in sorted(rng.choice(narrow, 6, replace=False)):
        ref = lc.lightcone_zz(r["n"], r["edges"], r["p"], r["g"][0], r["b"][0], int(e))[0]
        assert abs(r["zz"][e, 0, 0] - ref.real) < 1e-5 and abs(r["zz"][e, 0, 1] - ref.imag) < 1e-5


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
        assert abs(r["zz"][e, 0, 0] - zz[0]) < 1e-5 and abs(zz[1]) < 1e-10
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
    np.testing.assert_allclose(zz.cpu().numpy()[:, 0, 0], r["zz"][:, 0, 0], atol=2e-5, rtol=0)
    plan.close()


def _edge_energy_oracle(n, edges, p, g, b, e):
    return 0.5 * (1.0 - lc.lightcone_zz(n, edges, p, g, b, e)[0].real)


def test_gradient_of_narrow_edges_matches_oracle_differences(sliced_run):
    """dE_e/dgamma, dE_e/dbeta of single narrow edges (complex64 adjoint
    sweep, one-edge plans) against central differences (h = 1e-5) of the
    oracle's FP64 lightcone energy E_e = (1 - <ZZ>_e) / 2."""
    from paper_2106_15740_gb300.energy import EnergyPlan
    r = sliced_run
    n, edges, p, g, b = r["n"], r["edges"], r["p"], r["g"][0], r["b"][0]
    narrow = np.argsort(np.where(r["slices"] == 0, r["widths"], 99), kind="stable")[:2]
    assert r["widths"][narrow].max() <= 18
    h = 1e-5
    for e in (int(narrow[0]), int(narrow[1])):
        plan = EnergyPlan(n, edges, p, batch=1, dtype="c64", mode="persistent", gradient=True,
                          edge_range=(e, e + 1), device="cuda:0")
        _, grad = plan.energy(torch.tensor(r["g"], device="cuda:0"), torch.tensor(r["b"], device="cuda:0"),
                              grad=True)
        plan.check()
        grad = grad.cpu().numpy()[0]
        plan.close()
        ref = np.zeros(2 * p)
        for j in range(2 * p):
            gp, gm, bp, bm = g.copy(), g.copy(), b.copy(), b.copy()
            if j < p:
                gp[j] += h
                gm[j] -= h
            else:
                bp[j - p] += h
                bm[j - p] -= h
            ref[j] = (_edge_energy_oracle(n, edges, p, gp, bp, e) - _edge_energy_oracle(n, edges, p, gm, bm, e)) / (2 * h)
        np.testing.assert_allclose(grad, ref, atol=1e-5 * max(1.0, np.abs(ref).max()), rtol=0)


def test_gradient_of_a_sliced_edge_matches_complex128_differences(sliced_run):
    """A sliced edge (searched orders, budget 28): the complex64 adjoint
    sweep over its restricted networks against central differences
    (h = 1e-5) of the complex128 plan's energy of the same edge."""
    from paper_2106_15740_gb300.energy import EnergyPlan
    r = sliced_run
    n, edges, p = r["n"], r["edges"], r["p"]
    from paper_2106_15740_gb300 import binding as qb
    opt = qb.qt_plan_options_default()  # the whole graph's plan, only to find a sliced edge
    opt.dtype, opt.mode, opt.max_width, opt.slice, opt.order_trials = qb.QT_C64, qb.QT_MODE_PERSISTENT, 28, 1, 100
    full = qb.qt_plan_create(n, edges, p, opt)
    slices = qb.qt_plan_edge_slices(full, len(edges))
    qb.qt_plan_free(full)
    sliced = np.flatnonzero(slices > 0)
    e = int(sliced[np.argmin(slices[sliced])])
    kw = dict(batch=1, mode="persistent", max_width=28, slice=True, order_trials=100, edge_range=(e, e + 1),
              max_workspace=48 << 30, device="cuda:0")
    plan = EnergyPlan(n, edges, p, dtype="c64", gradient=True, **kw)
    assert plan.slices[0] > 0
    gd, bd = torch.tensor(r["g"], device="cuda:0"), torch.tensor(r["b"], device="cuda:0")
    _, grad = plan.energy(gd, bd, grad=True)
    plan.check()
    grad = grad.cpu().numpy()[0]
    plan.close()
    ref_plan = EnergyPlan(n, edges, p, dtype="c128", **kw)
    h = 1e-5
    ref = np.zeros(2 * p)
    for j in range(2 * p):
        d = torch.zeros((1, 2 * p), dtype=torch.float64, device="cuda:0")
        d[0, j] = h
        ep = ref_plan.energy(gd + d[:, :p], bd + d[:, p:])
        em = ref_plan.energy(gd - d[:, :p], bd - d[:, p:])
        ref[j] = float((ep - em).item()) / (2 * h)
    ref_plan.check()
    ref_plan.close()
    np.testing.assert_allclose(grad, ref, atol=1e-5 * max(1.0, np.abs(ref).max()), rtol=0)
