"""Chained steps (``fuse_chains``), checked on the host (no GPU).

In bucket elimination (§Tensor network contraction) a bucket's result is
eliminated next by the bucket of its first variable.  When that consumer has
no variable beyond the result and no other intermediate input, it only
contracts the result with its leaf factor, and a persistent plan on the
row-wide tiles evaluates them in one step (and up to three consumers in a
row, each eliminating the previous one's result): the result's rows meet the
consumer's leaf rows as they are formed and are never stored.  These tests rebuild the buckets of every planned network in Python
from the network's tensors and the plan's elimination order, select the
chains by that rule, and check the library's plan against them: the
algorithmic bytes drop by exactly the write and the read of each fused
result, the step count by one per absorbed consumer, and the schedule stays
race-free.
"""
import numpy as np
import pytest

from test_schedule import _data_bytes, _schedule, check_schedule
from workloads import random_regular_graph


def _plan(n, edges, p, B=64, dtype=None, fuse=1, gradient=0, mode=None, max_workspace=0, order_trials=0):
    from paper_2106_15740_gb300 import binding as qb
    opt = qb.qt_plan_options_default()
    opt.batch = B
    opt.dtype = qb.QT_C64 if dtype is None else dtype
    opt.mode = qb.QT_MODE_PERSISTENT if mode is None else mode
    opt.gradient = gradient
    opt.fuse_chains = fuse
    opt.max_workspace = max_workspace
    opt.order_trials = order_trials
    return qb.qt_plan_create(n, edges, p, opt)


def _buckets(tensors, order):
    """Buckets of (tensor variable lists, order): per bucket its output
    variables, its intermediate inputs (producer indices) and whether it has
    a leaf factor; plus each bucket's consumer."""
    pos = {v: i for i, v in enumerate(order)}
    pending = [[] for _ in order]
    for vs in tensors:
        vs = sorted(set(vs), key=pos.__getitem__)
        pending[pos[vs[0]]].append((vs, -1))
    out = []
    for i, v in enumerate(order):
        items = pending[i]
        U = sorted({v}.union(*[set(vs) for vs, _ in items]), key=pos.__getitem__)
        ints = [src for _, src in items if src >= 0]
        out.append(dict(S=U[1:], ints=ints, leaf=any(src < 0 for _, src in items), consumer=-1))
        for src in ints:
            out[src]["consumer"] = i
        if len(U) > 1:
            pending[pos[U[1]]].append((U[1:], i))
    return out


def _chains(bk, max_len, fan_in=None):
    """Greedy chains in execution order: from bucket b, c_1 = b's consumer and
    c_j = the consumer of c_(j-1), while c_j has no variable beyond its input
    (|U_(c_j)| = |S_(c_(j-1))|) and no other intermediate input, up to
    max_len consumers (and 8 input records: b's inputs plus one per consumer);
    a bucket absorbed into a chain starts none.  fan_in = (lo, hi): only a b
    with that many inputs starts one (the row-wide layout's rule)."""
    absorbed, chains = set(), []
    for i, b in enumerate(bk):
        if i in absorbed:
            continue
        n_in = len(b["ints"]) + (1 if b["leaf"] else 0)
        if fan_in is not None and not fan_in[0] <= n_in <= fan_in[1]:
            continue
        ch, cur = [], i
        while len(ch) < max_len and n_in + len(ch) < 8:
            c = bk[cur]["consumer"]
            if c < 0 or not bk[cur]["S"] or len(bk[c]["S"]) + 1 != len(bk[cur]["S"]) or bk[c]["ints"] != [cur]:
                break
            ch.append(c)
            absorbed.add(c)
            cur = c
        if ch:
            chains.append([i] + ch)
    return chains


def _network_tensors(n, edges, p, e):
    from paper_2106_15740_gb300 import binding as qb
    net = qb.qt_build_lightcone(n, edges, p, np.zeros(p), np.zeros(p), e)
    try:
        _, nt = qb.qt_network_info(net)
        out = []
        for t in range(nt):
            _, _, _, r, v = qb.qt_network_tensor(net, t)
            out.append([v[j] for j in range(r)])
        return out
    finally:
        qb.qt_network_free(net)


@pytest.mark.parametrize("max_len", [1, 2, 3])
@pytest.mark.parametrize("B,dtype_name,trials", [(64, "QT_C64", 0), (64, "QT_C64", 6), (34, "QT_C64", 0),
                                                 (32, "QT_C128", 0), (17, "QT_C64X2", 3), (1, "QT_C64", 4),
                                                 (1, "QT_C128", 0)])
def test_fused_plan_drops_each_fused_result(qtlib, B, dtype_name, trials, max_len):
    """(One angle set: chains of one consumer at most, whatever fuse_chains.
    Row-wide layout: complex64 only, from buckets of fan-in 2 or 3; complex128
    and float pairs there have no chained steps.)"""
    from paper_2106_15740_gb300 import binding as qb
    dtype = getattr(qb, dtype_name)
    es = {qb.QT_C64: 8, qb.QT_C128: 16, qb.QT_C64X2: 16}[dtype]
    n, p = 18, 3
    edges = random_regular_graph(n, 3, 51)
    plain = _plan(n, edges, p, B=B, dtype=dtype, fuse=0, order_trials=trials)
    fused = _plan(n, edges, p, B=B, dtype=dtype, fuse=max_len, order_trials=trials)
    try:
        s0, s1 = qb.qt_plan_stats(plain), qb.qt_plan_stats(fused)
        if B > 1 and dtype != qb.QT_C64:
            assert s0 == s1
            return
        saved, n_absorbed, longest = 0.0, 0, 0
        for e in range(len(edges)):
            order = list(qb.qt_plan_edge_order(fused, e))
            assert order == list(qb.qt_plan_edge_order(plain, e))
            bk = _buckets(_network_tensors(n, edges, p, e), order)
            for ch in _chains(bk, 1 if B == 1 else max_len, None if B == 1 else (2, 3)):
                n_absorbed += len(ch) - 1
                longest = max(longest, len(ch) - 1)
                # every result but the last one's is neither written nor read back
                saved += sum(2.0 * (1 << len(bk[k]["S"])) * B * es for k in ch[:-1])
        assert longest == (1 if B == 1 else max_len)
        assert s1["n_buckets"] == s0["n_buckets"] - n_absorbed
        assert s1["alg_bytes"] == s0["alg_bytes"] - saved
        assert s1["flops"] == s0["flops"]  # the same arithmetic
        assert qb.qt_plan_workspace_size(fused) <= qb.qt_plan_workspace_size(plain)
    finally:
        qb.qt_plan_free(plain)
        qb.qt_plan_free(fused)


@pytest.mark.parametrize("shared", [False, True])
def test_fused_schedule_is_race_free(qtlib, shared):
    """The fused step reads the first bucket's inputs and writes the
    consumer's output; with a workspace cap several networks share a slot."""
    from paper_2106_15740_gb300 import binding as qb
    from paper_2106_15740_gb300.schedule import bytes_by_rank
    n = 16
    edges = random_regular_graph(n, 3, 52)
    cap = 0
    if shared:
        full = _plan(n, edges, 3)
        cap = _data_bytes(full, es=8) // 2
        qb.qt_plan_free(full)
    plan = _plan(n, edges, 3, max_workspace=cap)
    try:
        units, depth, pairs, cross = check_schedule(*_schedule(plan))
        assert pairs > 0 and depth < units
        assert (cross > 0) == shared
        total = qb.qt_plan_stats(plan)["alg_bytes"]
        assert sum(bytes_by_rank(plan, 64, 8, 10).values()) == pytest.approx(total, rel=1e-12)
    finally:
        qb.qt_plan_free(plan)


@pytest.mark.parametrize("case", ["narrow_rows", "gradient", "per_bucket", "two_chunks"])
def test_no_fusion_outside_the_row_tiles(qtlib, case):
    """Gradient plans keep every result (the reverse sweep reads them); the
    per-bucket path, the narrow-row tiles (several rows per warp pass) and
    the two-chunk float-pair tile have no chained form: there the option
    changes nothing."""
    from paper_2106_15740_gb300 import binding as qb
    n = 14
    edges = random_regular_graph(n, 3, 53)
    kw = {"narrow_rows": dict(B=4), "gradient": dict(B=64, gradient=1),
          "per_bucket": dict(B=64, mode=qb.QT_MODE_PER_BUCKET),
          "two_chunks": dict(B=64, dtype=qb.QT_C64X2)}[case]
    a, b = _plan(n, edges, 2, fuse=0, **kw), _plan(n, edges, 2, fuse=1, **kw)
    try:
        assert qb.qt_plan_stats(a) == qb.qt_plan_stats(b)
    finally:
        qb.qt_plan_free(a)
        qb.qt_plan_free(b)


@pytest.mark.parametrize("value", [4, -1])
def test_fuse_option_is_validated(qtlib, value):
    from paper_2106_15740_gb300 import binding as qb
    opt = qb.qt_plan_options_default()
    assert opt.fuse_chains == 3
    opt.batch = 64
    opt.mode = qb.QT_MODE_PERSISTENT
    opt.fuse_chains = value
    with pytest.raises(qb.QTError) as ei:
        qb.qt_plan_create(8, random_regular_graph(8, 3, 39), 1, opt)
    assert ei.value.status == qb.QT_EINVAL


def test_bucket_bytes_count_every_bucket(qtlib):
    """EnergyPlan.bucket_bytes: the roofline's bytes, bucket by bucket, equal
    the unfused plan's algorithmic bytes whatever the chain length (a host
    plan; the workspace here is host memory and nothing is evaluated)."""
    from paper_2106_15740_gb300.energy import EnergyPlan
    n = 16
    edges = random_regular_graph(n, 3, 56)
    plans = [EnergyPlan(n, edges, 3, batch=64, dtype="c64", mode="persistent", device="cpu", fuse_chains=f)
             for f in (0, 1, 3)]
    try:
        unfused = plans[0].stats["alg_bytes"]
        assert plans[2].stats["alg_bytes"] < plans[1].stats["alg_bytes"] < unfused
        assert all(pl.bucket_bytes() == unfused for pl in plans)
    finally:
        for pl in plans:
            pl.close()
