"""Host-side logic of the C ABI, no GPU: symbol exports, network structure,
min-fill order parity with the oracle, argument validation."""
import re
from pathlib import Path

import numpy as np
import pytest

from oracle import lightcone as lc
from workloads import complete_graph, random_angles, random_regular_graph, workload

ROOT = Path(__file__).resolve().parent.parent


def test_library_exports_every_declared_symbol(qtlib):
    header = (ROOT / "include" / "qtensor.h").read_text()
    declared = set(re.findall(r"\b(qt_[a-z_]+)\s*\(", header))
    assert len(declared) >= 15
    for name in sorted(declared):
        assert hasattr(qtlib, name), name
    from paper_2106_15740_gb300 import binding as qb
    assert set(qb.EXPORTS) <= declared


def _lib_network(n, edges, p, g, b, e):
    from paper_2106_15740_gb300 import binding as qb
    net = qb.qt_build_lightcone(n, edges, p, g, b, e)
    nv, nt = qb.qt_network_info(net)
    tensors = [qb.qt_network_tensor(net, t) for t in range(nt)]
    order, width = qb.qt_order(net)
    qb.qt_network_free(net)
    return nv, tensors, list(order), width


@pytest.mark.parametrize("name,count", [("n16_p1", 24), ("n100_p3", 150), ("n100_p4", 40), ("n60_p4", 30)])
def test_network_and_order_match_oracle_bitwise(qtlib, name, count):
    """Same variables, same tensors (by kind/layer/side), same min-fill order
    and width as the oracle's independent implementation."""
    n, edges, p, g, b = workload(name)
    kinds = {0: "leaf", 1: "zz", 2: "mix", 3: "obs"}
    for e in range(0, len(edges), max(1, len(edges) // count)):
        nv, tensors, order, width = _lib_network(n, edges, p, g[0], b[0], e)
        net = lc.build_lightcone(n, edges, p, g[0], b[0], e)
        assert nv == net.n_vars
        mine = sorted((kinds[k], lay if k in (1, 2) else 0, "bra" if c else "ket",
                       tuple(v for v in vs if v >= 0)) for k, lay, c, r, vs in tensors)
        theirs = sorted((tag[0], tag[1] if tag[0] in ("zz", "mix") else 0, tag[2], tuple(vs))
                        for (vs, _), tag in zip(net.tensors, net.tags))
        assert mine == theirs
        o, w = lc.min_fill_order(net.n_vars, [vs for vs, _ in net.tensors])
        assert order == o and width == w


def test_plan_widths_and_stats(qtlib):
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, g, b = workload("n100_p3")
    opt = qb.qt_plan_options_default()
    opt.batch = 4
    opt.dtype = qb.QT_C64
    opt.mode = qb.QT_MODE_PERSISTENT
    plan = qb.qt_plan_create(n, edges, p, opt)
    st = qb.qt_plan_stats(plan)
    widths = qb.qt_plan_edge_widths(plan, len(edges))
    qb.qt_plan_free(plan)
    ref = [lc.min_fill_order(*(lambda net: (net.n_vars, [vs for vs, _ in net.tensors]))(
        lc.build_lightcone(n, edges, p, g[0], b[0], e)))[1] for e in range(len(edges))]
    assert list(widths) == ref
    assert st["n_edges"] == 150 and st["max_width"] == max(ref)
    assert st["alg_bytes"] > 0 and st["flops"] > 0


@pytest.mark.parametrize("bad", [
    dict(edges=[[0, 0]]), dict(edges=[[0, 5]]), dict(edges=[[0, 1], [1, 0]]), dict(edges=[[-1, 1]]),
])
def test_invalid_graphs_rejected(qtlib, bad):
    from paper_2106_15740_gb300 import binding as qb
    with pytest.raises(qb.QTError) as ei:
        qb.qt_build_lightcone(3, np.array(bad["edges"]), 1, [0.1], [0.2], 0)
    assert ei.value.status == qb.QT_EINVAL


def test_invalid_arguments_rejected(qtlib):
    from paper_2106_15740_gb300 import binding as qb
    edges = complete_graph(4)
    for kwargs in (dict(p=0, e=0, g=[0.1]), dict(p=1, e=6, g=[0.1]), dict(p=1, e=0, g=[np.nan])):
        with pytest.raises(qb.QTError) as ei:
            qb.qt_build_lightcone(4, edges, kwargs["p"], kwargs["g"], [0.2] * max(1, kwargs["p"]), kwargs["e"])
        assert ei.value.status == qb.QT_EINVAL
    opt = qb.qt_plan_options_default()
    opt.batch = 0
    with pytest.raises(qb.QTError):
        qb.qt_plan_create(4, edges, 1, opt)


def test_width_budget(qtlib):
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, g, b = workload("n100_p3")
    opt = qb.qt_plan_options_default()
    opt.max_width = 8
    with pytest.raises(qb.QTError) as ei:
        qb.qt_plan_create(n, edges, p, opt)
    assert ei.value.status == qb.QT_EWIDTH


def test_contract_rejects_bad_order(qtlib):
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, g, b = workload("n16_p1")
    net = qb.qt_build_lightcone(n, edges, p, g[0], b[0], 0)
    try:
        order, _ = qb.qt_order(net)
        order[1] = order[0]
        with pytest.raises(qb.QTError) as ei:
            qb.qt_contract_workspace_size(net, order, qb.QT_C128)
        assert ei.value.status == qb.QT_EINVAL
    finally:
        qb.qt_network_free(net)


def test_workspace_grows_with_batch_and_precision(qtlib):
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, g, b = workload("n16_p1")
    sizes = {}
    for B in (1, 8):
        for dt in (qb.QT_C64, qb.QT_C128):
            sizes[(B, dt)] = qb.qt_energy_workspace_size(n, edges, p, B, dt, 0)
    assert sizes[(8, qb.QT_C64)] > sizes[(1, qb.QT_C64)]
    assert sizes[(8, qb.QT_C128)] > sizes[(8, qb.QT_C64)]


def test_stall_hook_needs_a_waiting_task(qtlib):
    """Per-bucket plans have no queue, so there is nothing to stall."""
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, g, b = workload("n16_p1")
    opt = qb.qt_plan_options_default()
    plan = qb.qt_plan_create(n, edges, p, opt)
    try:
        with pytest.raises(qb.QTError) as ei:
            qb.qt_plan_inject_stall(plan, 1)
        assert ei.value.status == qb.QT_ESTATE
        qb.qt_plan_inject_stall(plan, 0)
        with pytest.raises(qb.QTError):
            qb.qt_plan_set_wait_limit(plan, 0)
    finally:
        qb.qt_plan_free(plan)


def test_gradient_plans_need_the_persistent_queue(qtlib):
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, g, b = workload("n16_p1")
    opt = qb.qt_plan_options_default()
    opt.gradient = 1
    opt.mode = qb.QT_MODE_PER_BUCKET
    with pytest.raises(qb.QTError) as ei:
        qb.qt_plan_create(n, edges, p, opt)
    assert ei.value.status == qb.QT_EINVAL


@pytest.mark.parametrize("name,max_width", [("n100_p3", 10), ("n60_p4", 23)])
def test_slicing_meets_the_width_budget(qtlib, name, max_width):
    """Without slicing a budget below an edge's width is an error; with it,
    exactly the edges above the budget get sliced variables and every planned
    width is within the budget."""
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, g, b = workload(name)
    opt = qb.qt_plan_options_default()
    plan = qb.qt_plan_create(n, edges, p, opt)
    w0 = qb.qt_plan_edge_widths(plan, len(edges))
    assert list(qb.qt_plan_edge_slices(plan, len(edges))) == [0] * len(edges)
    qb.qt_plan_free(plan)
    opt.max_width = max_width
    with pytest.raises(qb.QTError) as ei:
        qb.qt_plan_create(n, edges, p, opt)
    assert ei.value.status == qb.QT_EWIDTH
    opt.slice = 1
    plan = qb.qt_plan_create(n, edges, p, opt)
    try:
        w = qb.qt_plan_edge_widths(plan, len(edges))
        s = qb.qt_plan_edge_slices(plan, len(edges))
        st = qb.qt_plan_stats(plan)
    finally:
        qb.qt_plan_free(plan)
    assert st["n_edges"] == len(edges) and st["max_width"] <= max_width
    assert (w <= max_width).all()
    np.testing.assert_array_equal(s > 0, w0 > max_width)
    np.testing.assert_array_equal(w[w0 <= max_width], w0[w0 <= max_width])


def _plan_stats(name, batch=4, **kw):
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, g, b = workload(name)
    opt = qb.qt_plan_options_default()
    opt.batch = batch
    opt.dtype = qb.QT_C64
    for k, v in kw.items():
        setattr(opt, k, v)
    plan = qb.qt_plan_create(n, edges, p, opt)
    try:
        return qb.qt_plan_stats(plan), qb.qt_plan_edge_widths(plan, len(edges)), qb.qt_plan_edge_bytes(plan, len(edges))
    finally:
        qb.qt_plan_free(plan)


def test_order_search_is_never_wider_or_costlier_than_min_fill(qtlib):
    """The randomised greedy search keeps min-fill among its candidates and
    only accepts orders no wider, so per edge the width never grows and the
    planned bytes fall on the wide 100-vertex p = 4 graph."""
    st0, w0, c0 = _plan_stats("n100_p4")
    st1, w1, c1 = _plan_stats("n100_p4", order_trials=30, order_seed=3)
    assert (w1 <= w0).all()
    assert st1["alg_bytes"] < 0.6 * st0["alg_bytes"]
    assert st1["n_edges"] == st0["n_edges"] == 150


def test_order_search_is_deterministic_per_seed(qtlib):
    from paper_2106_15740_gb300 import binding as qb
    a = _plan_stats("n60_p4", order_trials=10, order_seed=7)
    b = _plan_stats("n60_p4", order_trials=10, order_seed=7)
    c = _plan_stats("n60_p4", order_trials=10, order_seed=8)
    np.testing.assert_array_equal(a[2], b[2])
    assert a[0]["alg_bytes"] == b[0]["alg_bytes"]
    assert not np.array_equal(a[2], c[2])
    opt = qb.qt_plan_options_default()
    n, edges, p, g, bb = workload("n16_p1")
    for bad in (dict(order_trials=-1), dict(order_tau=float("nan"))):
        o = qb.qt_plan_options_default()
        for k, v in bad.items():
            setattr(o, k, v)
        with pytest.raises(qb.QTError) as ei:
            qb.qt_plan_create(n, edges, p, o)
        assert ei.value.status == qb.QT_EINVAL


def test_single_network_workspace_for_every_edge(qtlib):
    """The single-network path plans one network whose graph edge id is not
    its index in the plan."""
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, g, b = workload("n100_p3")
    for e in (0, 1, 77, 149):
        net = qb.qt_build_lightcone(n, edges, p, g[0], b[0], e)
        try:
            order, _ = qb.qt_order(net)
            for dt in (qb.QT_C64, qb.QT_C128):
                assert qb.qt_contract_workspace_size(net, order, dt) > 0
        finally:
            qb.qt_network_free(net)


def test_checkpoint_segments_add_recompute_traffic(qtlib):
    """Gradient plans with a checkpoint budget re-run forward steps: more
    steps and algorithmic bytes than the unsegmented plan; a budget larger
    than every network keeps the unsegmented plan."""
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, _, _ = workload("n100_p3")
    stats = {}
    for cb in (0, 1 << 40, 1 << 12):
        opt = qb.qt_plan_options_default()
        opt.batch, opt.dtype, opt.mode, opt.gradient = 1, qb.QT_C64, qb.QT_MODE_PERSISTENT, 1
        opt.checkpoint_bytes = cb
        pl = qb.qt_plan_create(n, np.asarray(edges, np.int32), p, opt)
        stats[cb] = (qb.qt_plan_stats(pl), qb.qt_plan_workspace_size(pl))
        qb.qt_plan_free(pl)
    assert stats[1 << 40] == stats[0]
    assert stats[1 << 12][0]["n_buckets"] > stats[0][0]["n_buckets"]
    assert stats[1 << 12][0]["alg_bytes"] > stats[0][0]["alg_bytes"]
    opt = qb.qt_plan_options_default()
    opt.checkpoint_bytes = -1
    with pytest.raises(qb.QTError):
        qb.qt_plan_create(n, np.asarray(edges, np.int32), p, opt)


def test_amplitude_plans_validate_and_size(qtlib):
    """Amplitude networks: one per bitstring, no gradient, 0/1 bytes only;
    on a 40-vertex p = 3 graph the searched order is narrower than min-fill."""
    from paper_2106_15740_gb300 import binding as qb
    n, p = 40, 3
    edges = random_regular_graph(n, 3, 53)
    bits = np.zeros((2, n), dtype=np.uint8)
    widths = {}
    for trials in (0, 50):
        opt = qb.qt_plan_options_default()
        opt.mode, opt.order_trials = qb.QT_MODE_PERSISTENT, trials
        pl = qb.qt_amplitude_plan_create(n, edges, p, bits, opt)
        widths[trials] = list(qb.qt_plan_edge_widths(pl, 2))
        assert qb.qt_plan_stats(pl)["n_edges"] == 2
        qb.qt_plan_free(pl)
    assert max(widths[50]) <= max(widths[0])
    opt = qb.qt_plan_options_default()
    bad = bits.copy()
    bad[0, 3] = 2
    with pytest.raises(qb.QTError):
        qb.qt_amplitude_plan_create(n, edges, p, bad, opt)
    opt.gradient, opt.mode = 1, qb.QT_MODE_PERSISTENT
    with pytest.raises(qb.QTError):
        qb.qt_amplitude_plan_create(n, edges, p, bits, opt)


@pytest.mark.parametrize("n,p", [(20, 1), (20, 3), (40, 2)])
def test_representation_variable_counts(qtlib, n, p):
    """Free variables of the amplitude network per representation (outputs
    projected): ZZ+diagonal n p; ZZ adds two per ZZ gate; diagonal keeps the
    Z rotations and CNOT controls but opens one index per CNOT target and
    per Hadamard; default opens one per gate index."""
    from paper_2106_15740_gb300 import binding as qb
    edges = random_regular_graph(n, 3, 1)
    m = len(edges)
    expect = {qb.QT_REP_ZZ_DIAGONAL: n * p, qb.QT_REP_ZZ: n * p + 2 * m * p,
              qb.QT_REP_DIAGONAL: p * (2 * n + 2 * m), qb.QT_REP_DEFAULT: p * (3 * n + 5 * m)}
    for rep, nv in expect.items():
        assert qb.qt_representation_cost(n, edges, p, rep)[0] == nv


def test_zz_diagonal_representation_is_the_amplitude_network(qtlib):
    """The cost study's ZZ + diagonal structure is the interaction graph of the
    amplitude plans: same min-fill width."""
    from paper_2106_15740_gb300 import binding as qb
    for n, p, seed in ((30, 2, 3), (40, 3, 4)):
        edges = random_regular_graph(n, 3, seed)
        _, w, _ = qb.qt_representation_cost(n, edges, p, qb.QT_REP_ZZ_DIAGONAL)
        opt = qb.qt_plan_options_default()
        opt.mode = qb.QT_MODE_PERSISTENT
        pl = qb.qt_amplitude_plan_create(n, edges, p, np.zeros((1, n), np.uint8), opt)
        assert int(qb.qt_plan_edge_widths(pl, 1)[0]) == w
        qb.qt_plan_free(pl)


def test_simplifications_lower_width_and_cost_at_depth(qtlib):
    """At p = 3 on 40 vertices the diagonal and ZZ simplifications cut the
    width and cost by orders of magnitude (the paper's Table 1 regime)."""
    from paper_2106_15740_gb300 import binding as qb
    from paper_2106_15740_gb300.cost_study import LAPTOP_BYTES, fits
    edges = random_regular_graph(40, 3, 0)
    r = {rep: qb.qt_representation_cost(40, edges, 3, rep, 10, 0) for rep in range(4)}
    assert r[qb.QT_REP_ZZ_DIAGONAL][1] <= r[qb.QT_REP_DIAGONAL][1] < r[qb.QT_REP_DEFAULT][1]
    assert r[qb.QT_REP_DEFAULT][2] - r[qb.QT_REP_ZZ_DIAGONAL][2] >= 10  # >= 1000x fewer FLOPs
    assert fits(r[qb.QT_REP_ZZ_DIAGONAL][1], LAPTOP_BYTES) and not fits(r[qb.QT_REP_DEFAULT][1], LAPTOP_BYTES)
    with pytest.raises(qb.QTError):
        qb.qt_representation_cost(40, edges, 3, 7)


def _oracle_bucket_flops(n, edges, p, e):
    """Real FLOPs of bucket elimination (per bucket 6 (k - 1)
    2^|U| for the products of its k inputs at both values of the eliminated
    variable, plus 2^|U| for the sum over it), counted on the oracle's own
    network and min-fill order, with a bucket's leaf tensors taken as one
    input (the library multiplies them into one leaf factor before the
    launch)."""
    net = lc.build_lightcone(n, edges, p, np.zeros(p), np.zeros(p), e)
    tvars = [vs for vs, _ in net.tensors]
    order, _ = lc.min_fill_order(net.n_vars, tvars)
    live = [(frozenset(vs), True) for vs in tvars]  # (variables, is a leaf)
    flops = 0
    for v in order:
        bucket = [t for t in live if v in t[0]]
        live = [t for t in live if v not in t[0]]
        union = frozenset().union(*[t[0] for t in bucket])
        k = sum(1 for t in bucket if not t[1]) + (1 if any(t[1] for t in bucket) else 0)
        flops += 2 ** len(union) * 6 * (k - 1) + 2 ** len(union)
        live.append((union - {v}, False))
    return flops


@pytest.mark.parametrize("name", ["n16_p1", "n100_p3"])
def test_plan_flops_match_oracle_buckets(qtlib, name):
    """qt_plan_stats' FLOPs (the complex128 roofline's numerator) against a
    count over the oracle's buckets, per edge, and B times that for B angle
    sets."""
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, _, _ = workload(name)
    for e in range(0, len(edges), max(1, len(edges) // 6)):
        for B in (1, 3):
            opt = qb.qt_plan_options_default()
            opt.batch, opt.dtype = B, qb.QT_C128
            opt.edge_begin, opt.edge_end = e, e + 1
            plan = qb.qt_plan_create(n, edges, p, opt)
            try:
                assert qb.qt_plan_stats(plan)["flops"] == B * _oracle_bucket_flops(n, edges, p, e)
            finally:
                qb.qt_plan_free(plan)


def _oracle_bucket_elems(n, edges, p, e):
    """Complex elements moved per angle set, counted on the oracle's buckets
    (min-fill order): forward, every bucket's intermediate inputs read and
    its result written; reverse sweep, one adjoint step per
    input of every bucket (the leaf factor, a bucket's leaf tensors taken as
    one, included), each reading the output adjoint and the other
    intermediate inputs and writing its target."""
    net = lc.build_lightcone(n, edges, p, np.zeros(p), np.zeros(p), e)
    tvars = [vs for vs, _ in net.tensors]
    order, _ = lc.min_fill_order(net.n_vars, tvars)
    live = [(frozenset(vs), True) for vs in tvars]  # (variables, is a leaf)
    fwd = rev = 0
    for v in order:
        bucket = [t for t in live if v in t[0]]
        live = [t for t in live if v not in t[0]]
        union = frozenset().union(*[t[0] for t in bucket])
        out = len(union) - 1
        inputs = [(len(t[0]), True) for t in bucket if not t[1]]  # (rank, intermediate)
        leaves = [t[0] for t in bucket if t[1]]
        if leaves:
            inputs.append((len(frozenset().union(*leaves)), False))
        fwd += 2 ** out + sum(2 ** r for r, inter in inputs if inter)
        for i, (ri, _) in enumerate(inputs):
            rev += 2 ** out + 2 ** ri + sum(2 ** r for j, (r, inter) in enumerate(inputs) if j != i and inter)
        live.append((union - {v}, False))
    return fwd, rev


@pytest.mark.parametrize("name", ["n16_p1", "n100_p3"])
def test_plan_bytes_match_oracle_buckets(qtlib, name):
    """qt_plan_stats' algorithmic bytes (the rooflines' numerators) of energy
    and gradient plans against a count over the oracle's buckets, per edge,
    for complex128 (16 bytes per element) and complex64 (8)."""
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, _, _ = workload(name)
    for e in range(0, len(edges), max(1, len(edges) // 6)):
        fwd, rev = _oracle_bucket_elems(n, edges, p, e)
        for dtype, es in ((qb.QT_C128, 16), (qb.QT_C64, 8)):
            for grad in (0, 1):
                opt = qb.qt_plan_options_default()
                opt.batch, opt.dtype, opt.mode, opt.gradient = 2, dtype, qb.QT_MODE_PERSISTENT, grad
                opt.fuse_chains = 0
                opt.edge_begin, opt.edge_end = e, e + 1
                plan = qb.qt_plan_create(n, edges, p, opt)
                try:
                    assert qb.qt_plan_stats(plan)["alg_bytes"] == 2 * es * (fwd + rev * grad)
                finally:
                    qb.qt_plan_free(plan)
