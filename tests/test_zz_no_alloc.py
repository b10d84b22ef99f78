"""The allocation-free entry point, qt_plan_energy_static.

It exists for callers that may not allocate device memory while they run
(a service holding a fixed device-memory budget, a plug-in whose host owns
all device allocations): the plan's scratch space lives in a device array
built into the library instead of a caller workspace.  This test compares
it, through the C ABI, with the workspace entry point qt_plan_energy on two
calls in a row (the second with other angles, so stale contents of the
shared array would show; the second call reuses the descriptors the first
one uploaded), and on calls that alternate between two plans (each switch
uploads the other plan's descriptors again), within the complex128
tolerance of the parity tests.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import random_angles, workload

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib(qtlib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return qtlib


def _plan(name, batch, dtype, mode):
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, _, _ = workload(name)
    opt = qb.qt_plan_options_default()
    opt.batch = batch
    opt.dtype = dtype
    opt.mode = mode
    return qb.qt_plan_create(n, edges, p, opt), len(edges), p


def test_static_scratch_matches_workspace_call_twice():
    from paper_2106_15740_gb300 import binding as qb
    plan, n_edges, p = _plan("n100_p3", 2, qb.QT_C128, qb.QT_MODE_PERSISTENT)
    try:
        assert qb.qt_plan_workspace_size(plan) <= qb.qt_static_scratch_bytes()
        ws_bytes = qb.qt_plan_workspace_size(plan)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda:0")
        stream = torch.cuda.current_stream().cuda_stream
        for seed in (5, 6):
            g, b = random_angles(2, p, seed)
            gd = torch.tensor(g, device="cuda:0")
            bd = torch.tensor(b, device="cuda:0")
            e_ref = torch.empty(2, dtype=torch.float64, device="cuda:0")
            zz_ref = torch.empty((n_edges, 2, 2), dtype=torch.float64, device="cuda:0")
            qb.qt_plan_energy(plan, gd.data_ptr(), bd.data_ptr(), e_ref.data_ptr(), zz_ref.data_ptr(), 0,
                              ws.data_ptr(), ws_bytes, stream)
            e_st = torch.full((2,), np.nan, dtype=torch.float64, device="cuda:0")
            zz_st = torch.full((n_edges, 2, 2), np.nan, dtype=torch.float64, device="cuda:0")
            qb.qt_plan_energy_static(plan, gd.data_ptr(), bd.data_ptr(), e_st.data_ptr(), zz_st.data_ptr(), stream)
            qb.qt_plan_check(plan, stream)
            np.testing.assert_allclose(e_st.cpu().numpy(), e_ref.cpu().numpy(), atol=TOL * n_edges, rtol=0)
            np.testing.assert_allclose(zz_st.cpu().numpy(), zz_ref.cpu().numpy(), atol=TOL, rtol=0)
    finally:
        qb.qt_plan_free(plan)


def _compare(qb, plan, n_edges, p, seed):
    stream = torch.cuda.current_stream().cuda_stream
    ws_bytes = qb.qt_plan_workspace_size(plan)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda:0")
    g, b = random_angles(2, p, seed)
    gd = torch.tensor(g, device="cuda:0")
    bd = torch.tensor(b, device="cuda:0")
    e_ref = torch.empty(2, dtype=torch.float64, device="cuda:0")
    zz_ref = torch.empty((n_edges, 2, 2), dtype=torch.float64, device="cuda:0")
    qb.qt_plan_energy(plan, gd.data_ptr(), bd.data_ptr(), e_ref.data_ptr(), zz_ref.data_ptr(), 0,
                      ws.data_ptr(), ws_bytes, stream)
    e_st = torch.full((2,), np.nan, dtype=torch.float64, device="cuda:0")
    zz_st = torch.full((n_edges, 2, 2), np.nan, dtype=torch.float64, device="cuda:0")
    qb.qt_plan_energy_static(plan, gd.data_ptr(), bd.data_ptr(), e_st.data_ptr(), zz_st.data_ptr(), stream)
    qb.qt_plan_check(plan, stream)
    np.testing.assert_allclose(e_st.cpu().numpy(), e_ref.cpu().numpy(), atol=TOL * n_edges, rtol=0)
    np.testing.assert_allclose(zz_st.cpu().numpy(), zz_ref.cpu().numpy(), atol=TOL, rtol=0)


def test_static_scratch_alternating_plans():
    """Plans A, B, A, B: every switch must bring the other plan's
    descriptors back into the shared array."""
    from paper_2106_15740_gb300 import binding as qb
    a, na, pa = _plan("n100_p3", 2, qb.QT_C128, qb.QT_MODE_PERSISTENT)
    b, nb, pb = _plan("n16_p1", 2, qb.QT_C128, qb.QT_MODE_PERSISTENT)
    try:
        for k, (plan, n_edges, p) in enumerate([(a, na, pa), (b, nb, pb), (a, na, pa), (b, nb, pb)]):
            _compare(qb, plan, n_edges, p, 40 + k)
    finally:
        qb.qt_plan_free(a)
        qb.qt_plan_free(b)


def test_static_scratch_rejects_plans_above_its_size():
    from paper_2106_15740_gb300 import binding as qb
    plan, _, p = _plan("n100_p4", 64, qb.QT_C64, qb.QT_MODE_PERSISTENT)
    try:
        assert qb.qt_plan_workspace_size(plan) > qb.qt_static_scratch_bytes()
        g = torch.zeros((64, p), dtype=torch.float64, device="cuda:0")
        e = torch.empty(64, dtype=torch.float64, device="cuda:0")
        with pytest.raises(qb.QTError) as ei:
            qb.qt_plan_energy_static(plan, g.data_ptr(), g.data_ptr(), e.data_ptr(), 0,
                                     torch.cuda.current_stream().cuda_stream)
        assert ei.value.status == qb.QT_ENOMEM
    finally:
        qb.qt_plan_free(plan)


def test_static_scratch_chained_plan():
    """A plan with chained steps (complex64, one angle set: its kernel is the
    chained-step instantiation) gives the workspace call's values bit for bit
    through the static array."""
    from paper_2106_15740_gb300 import binding as qb
    plan, n_edges, p = _plan("n100_p3", 1, qb.QT_C64, qb.QT_MODE_PERSISTENT)
    try:
        assert qb.qt_plan_tasks(plan)["kind"].size > 0
        ws_bytes = qb.qt_plan_workspace_size(plan)
        assert ws_bytes <= qb.qt_static_scratch_bytes()
        stream = torch.cuda.current_stream().cuda_stream
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda:0")
        g, b = random_angles(1, p, 9)
        gd = torch.tensor(g, device="cuda:0")
        bd = torch.tensor(b, device="cuda:0")
        out = []
        for static in (False, True):
            e = torch.full((1,), np.nan, dtype=torch.float64, device="cuda:0")
            zz = torch.full((n_edges, 1, 2), np.nan, dtype=torch.float64, device="cuda:0")
            if static:
                qb.qt_plan_energy_static(plan, gd.data_ptr(), bd.data_ptr(), e.data_ptr(), zz.data_ptr(), stream)
            else:
                qb.qt_plan_energy(plan, gd.data_ptr(), bd.data_ptr(), e.data_ptr(), zz.data_ptr(), 0,
                                  ws.data_ptr(), ws_bytes, stream)
            qb.qt_plan_check(plan, stream)
            out.append((e.cpu().numpy(), zz.cpu().numpy()))
        assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    finally:
        qb.qt_plan_free(plan)
