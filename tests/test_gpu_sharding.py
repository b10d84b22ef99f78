"""Edge-range shards on the GPU: the partial energies and gradients of the
ranges of a cost-balanced partition sum to the whole-graph plan's values
(the shards run one after another in this process; the sum is what the
all-reduce of a multi-GPU run computes)."""
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


@pytest.mark.parametrize("world", [2, 3])
def test_shard_partials_sum_to_the_whole_graph(world):
    from paper_2106_15740_gb300.energy import EnergyPlan
    from paper_2106_15740_gb300.sharding import edge_costs, partition
    n, edges, p, g, b = workload("n60_p4", batch=2)
    gd, bd = torch.tensor(g, device="cuda:0"), torch.tensor(b, device="cuda:0")
    full = EnergyPlan(n, edges, p, batch=2, dtype="c128", mode="persistent", gradient=True, device="cuda:0")
    e_full, g_full = full.energy(gd, bd, grad=True)
    full.check()
    ranges = partition(edge_costs(n, edges, p, batch=2, dtype="c128"), world)
    e_sum = torch.zeros_like(e_full)
    g_sum = torch.zeros_like(g_full)
    for a, e1 in ranges:
        shard = EnergyPlan(n, edges, p, batch=2, dtype="c128", mode="persistent", gradient=True,
                           edge_range=(a, e1), device="cuda:0")
        e, gr = shard.energy(gd, bd, grad=True)
        shard.check()
        e_sum += e
        g_sum += gr
        shard.close()
    np.testing.assert_allclose(e_sum.cpu().numpy(), e_full.cpu().numpy(), atol=1e-10, rtol=0)
    np.testing.assert_allclose(g_sum.cpu().numpy(), g_full.cpu().numpy(), atol=1e-9, rtol=0)


def test_sharded_energy_single_rank_equals_plan():
    from paper_2106_15740_gb300.energy import EnergyPlan
    from paper_2106_15740_gb300.sharding import ShardedEnergy
    n, edges, p, g, b = workload("n100_p3", batch=2)
    gd, bd = torch.tensor(g, device="cuda:0"), torch.tensor(b, device="cuda:0")
    sh = ShardedEnergy(n, edges, p, batch=2, dtype="c128", mode="persistent", gradient=True, device="cuda:0")
    assert sh.ranges == [(0, len(edges))]
    e, gr = sh.energy(gd, bd, grad=True)
    sh.check()
    ref = EnergyPlan(n, edges, p, batch=2, dtype="c128", mode="persistent", gradient=True, device="cuda:0")
    e0, g0 = ref.energy(gd, bd, grad=True)
    # the reverse sweep accumulates with atomics: equal up to rounding order
    np.testing.assert_allclose(e.cpu().numpy(), e0.cpu().numpy(), atol=1e-12, rtol=0)
    np.testing.assert_allclose(gr.cpu().numpy(), g0.cpu().numpy(), atol=1e-10, rtol=0)
