"""GPU: chained steps (``fuse_chains``) are bit-identical to separate steps.

A fused step forms a bucket's two result rows w = 0, 1 exactly as the
bucket's own step does, and contracts them with the consumer's leaf rows in
the consumer's own operand order (result first, then the leaf, then the sum
over w), so every edge value and energy equals the unfused plan bit for bit.
The unfused plans are pinned against the oracle elsewhere.  Cases: the
row-wide complex64 tile with two angle sets per lane (64 and 34 angle sets),
the one-angle-set pair tiles of all three precisions (one consumer per step,
combined across lanes), searched orders, and networks sharing workspace
slots under a cap; complex128 and float pairs on the row-wide layout have no
chained steps (the option changes nothing there).
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


def _run(plan, g, b):
    e, zz = plan.energy(torch.tensor(g, device="cuda:0"), torch.tensor(b, device="cuda:0"), edge_zz=True)
    plan.check()
    return e.cpu().numpy(), zz.cpu().numpy()


@pytest.mark.parametrize("wl,dtype,batch,trials,capped", [
    ("n100_p3", "c64", 64, 20, False),
    ("n60_p4", "c64", 34, 20, False),
    ("n100_p3", "c128", 32, 0, False),
    ("n100_p3", "c64x2", 17, 5, False),
    ("n100_p3", "c64", 64, 20, True),
    ("n60_p4", "c64", 1, 100, False),
    ("n100_p3", "c128", 1, 0, False),
    ("n100_p3", "c64x2", 1, 5, False),
])
def test_fused_equals_unfused_bitwise(wl, dtype, batch, trials, capped):
    """Chains of up to 1, 2 and 3 consumers per step against none."""
    from paper_2106_15740_gb300 import binding as qb
    from paper_2106_15740_gb300.energy import DTYPES, EnergyPlan
    n, edges, p, g, b = workload(wl, batch=batch)
    cap = 0
    if capped:  # a third of the unfused plan's workspace: several networks per slot
        opt = qb.qt_plan_options_default()
        opt.batch, opt.dtype, opt.mode, opt.order_trials = batch, DTYPES[dtype], qb.QT_MODE_PERSISTENT, trials
        opt.fuse_chains = 0
        probe = qb.qt_plan_create(n, edges, p, opt)
        cap = qb.qt_plan_workspace_size(probe) // 3
        qb.qt_plan_free(probe)
    out, stats = {}, {}
    for fuse in (0, 1, 2, 3):
        plan = EnergyPlan(n, edges, p, batch=batch, dtype=dtype, mode="persistent", device="cuda:0",
                          order_trials=trials, fuse_chains=fuse, max_workspace=cap)
        out[fuse] = _run(plan, g, b)
        stats[fuse] = plan.stats
        plan.close()
        torch.cuda.empty_cache()
    for fuse in (1, 2, 3):
        if batch > 1 and dtype != "c64":  # row-wide layout: chained steps in complex64 only
            assert stats[fuse] == stats[0]
        elif batch == 1 and fuse > 1:  # one angle set: one consumer per step at most
            assert stats[fuse] == stats[1]
        else:
            assert stats[fuse]["alg_bytes"] < stats[fuse - 1]["alg_bytes"]
            assert stats[fuse]["n_buckets"] < stats[fuse - 1]["n_buckets"]
        assert np.array_equal(out[fuse][1], out[0][1]), fuse
        assert np.array_equal(out[fuse][0], out[0][0]), fuse
