"""Queue tracing of the persistent launch (measurement hook).

Every queue task gets (claimed, ready, done) device-clock readings in order
and the SM / warp that ran it; tracing does not change the results.
"""
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


@pytest.mark.parametrize("batch", [64, 1])
def test_trace_covers_every_task_in_order(batch):
    from paper_2106_15740_gb300.energy import EnergyPlan
    n, edges, p, g, b = workload("n100_p3", batch=batch)
    plan = EnergyPlan(n, edges, p, batch=batch, dtype="c64", mode="persistent", device="cuda:0")
    gd, bd = torch.tensor(g, device="cuda:0"), torch.tensor(b, device="cuda:0")
    e0 = plan.energy(gd, bd).clone()
    tr, tasks = plan.trace(gd, bd)
    e1 = plan.energy(gd, bd)
    plan.check()
    assert torch.equal(e0, e1)
    n_tasks = len(tasks["step"])
    assert tr.shape == (n_tasks, 4)
    claim, ready, done = (tr[:, i].astype(np.int64) for i in range(3))
    assert np.all(claim > 0)
    assert np.all(claim <= ready) and np.all(ready <= done)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert np.all((tr[:, 3] >> 16) < sms) and np.all((tr[:, 3] & 0xFFFF) < 8)
    assert np.all(tasks["edge"] >= 0) and np.all(tasks["edge"] < len(edges))
    assert set(np.unique(tasks["n_in"])) <= set(range(1, 9))
    plan.close()


def test_trace_rejects_a_short_buffer_and_per_bucket_plans():
    from paper_2106_15740_gb300 import binding as qb
    from paper_2106_15740_gb300.energy import EnergyPlan
    n, edges, p, g, b = workload("n16_p1")
    plan = EnergyPlan(n, edges, p, batch=1, dtype="c128", mode="persistent", device="cuda:0")
    need = qb.qt_plan_trace_size(plan.plan)
    buf = torch.zeros(need, dtype=torch.uint8, device="cuda:0")
    with pytest.raises(qb.QTError):
        qb.qt_plan_set_trace(plan.plan, buf.data_ptr(), need - 8)
    plan.close()
    plan = EnergyPlan(n, edges, p, batch=1, dtype="c128", mode="per_bucket", device="cuda:0")
    with pytest.raises(qb.QTError):
        qb.qt_plan_set_trace(plan.plan, buf.data_ptr(), need)
    plan.close()
