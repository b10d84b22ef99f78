"""Failure detection without a GPU fault: a bounded dependency wait that runs
out must stop every warp, report QT_ETIMEOUT through qt_plan_check, and leave
the CUDA context usable.  The fault is injected on the host: the uploaded
tile count of one awaited step is made unreachable (nothing ever sets it)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(qtlib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return qtlib


@pytest.mark.parametrize("gradient", [False, True])
def test_stalled_dependency_times_out_and_context_survives(gradient):
    from paper_2106_15740_gb300 import binding as qb
    from paper_2106_15740_gb300.energy import EnergyPlan
    n, edges, p, g, b = workload("n100_p3")
    plan = EnergyPlan(n, edges, p, batch=1, dtype="c64", mode="persistent", group_rows=-1,
                      gradient=gradient, device="cuda:0")
    gd, bd = torch.tensor(g, device="cuda:0"), torch.tensor(b, device="cuda:0")
    ref = plan.energy(gd, bd, grad=gradient)
    plan.check()
    ref = [t.cpu().numpy() for t in (ref if gradient else (ref,))]

    qb.qt_plan_set_wait_limit(plan.plan, 1 << 14)
    qb.qt_plan_inject_stall(plan.plan, 1)
    plan.energy(gd, bd, grad=gradient)
    with pytest.raises(qb.QTError) as ei:
        plan.check()
    assert ei.value.status == qb.QT_ETIMEOUT

    qb.qt_plan_inject_stall(plan.plan, 0)
    qb.qt_plan_set_wait_limit(plan.plan, 1 << 22)
    again = plan.energy(gd, bd, grad=gradient)
    plan.check()
    again = [t.cpu().numpy() for t in (again if gradient else (again,))]
    np.testing.assert_array_equal(again[0], ref[0])
    if gradient:  # atomics make the adjoint sums order-dependent in the last bits
        np.testing.assert_allclose(again[1], ref[1], atol=1e-4 * max(1.0, np.abs(ref[1]).max()), rtol=0)
    # an unrelated allocation and kernel still work on this context
    x = torch.ones(1 << 20, device="cuda:0")
    assert float(x.sum().item()) == float(1 << 20)
