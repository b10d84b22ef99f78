"""The persistent queue's dependency graph, checked on the host (no GPU).

A persistent plan lets a step start once the steps that last wrote what it
reads, and the last writer and readers of what it writes, are done (bucket
elimination forms a tree, §Tensor network contraction; the arena reuses
released space), instead of chaining every step of a workspace slot.  That is
only safe if every two steps that touch the same workspace elements, one of
them writing, are ordered by the dependency graph as they are in queue order.
These tests take the schedule the library reports (``qt_plan_schedule``: the
element ranges each step reads and writes, its dependency list) and check
exactly that, pair by pair, together with: every dependency lies earlier in
the queue (a persistent kernel whose warps claim tasks in queue order cannot
then wait forever), and the dependency paths are shorter than the chain.
"""
import numpy as np
import pytest

from workloads import random_regular_graph


def _plan(n, edges, p, B=4, chain=0, group_rows=0, max_workspace=0, order_trials=0, dtype=None, queue_order=1,
          by_rank=None):
    from paper_2106_15740_gb300 import binding as qb
    opt = qb.qt_plan_options_default()
    opt.batch = B
    opt.dtype = qb.QT_C64 if dtype is None else dtype
    opt.mode = qb.QT_MODE_PERSISTENT
    opt.chain_steps = chain
    opt.group_rows = group_rows
    opt.max_workspace = max_workspace
    opt.order_trials = order_trials
    opt.queue_order = queue_order
    for r, t in (by_rank or {}).items():
        opt.chunk_tiles_by_rank[r] = t
    return qb.qt_plan_create(n, edges, p, opt)


def _data_bytes(plan, es=8):
    """Bytes of a plan's data region up to the last element any step touches."""
    from paper_2106_15740_gb300 import binding as qb
    return int(qb.qt_plan_schedule(plan)["acc_hi"].max()) * es


def _schedule(plan):
    from paper_2106_15740_gb300 import binding as qb
    sch = qb.qt_plan_schedule(plan)
    tasks = qb.qt_plan_tasks(plan)
    return sch, tasks


def check_schedule(sch, tasks):
    """Asserts the schedule is race-free; returns (units, longest dependency
    path in units, ordered conflicting pairs, of them between two edges' networks)."""
    unit = sch["unit"]
    n = len(unit)
    # queue position of each unit (first task that runs it)
    qpos = np.full(n, -1, dtype=np.int64)
    for t, s in enumerate(tasks["step"]):
        if qpos[s] < 0:
            qpos[s] = t
    units = np.nonzero(unit == np.arange(n))[0]
    assert (qpos[units] >= 0).all()
    order = units[np.argsort(qpos[units], kind="stable")]
    # ancestors of each unit (python ints as bitsets over unit ranks), in queue order
    rank = {int(u): i for i, u in enumerate(order)}
    anc = [0] * len(order)
    depth = [0] * len(order)
    for i, u in enumerate(order):
        d0, dc = int(sch["dep_first"][u]), int(sch["dep_count"][u])
        a, dp = 0, 0
        for d in sch["deps"][d0:d0 + dc]:
            du = int(unit[d])
            # a dependency is the last step of its unit (its done counter)
            assert du != u
            last = du + int((unit[du:] == du).sum()) - 1
            assert int(d) == last, "a dependency must name the last step of its group"
            j = rank[du]
            assert j < i, "dependency later in the queue than the step waiting for it"
            a |= anc[j] | (1 << j)
            dp = max(dp, depth[j] + 1)
        anc[i] = a
        depth[i] = dp
    step_rank = np.array([rank[int(u)] for u in unit])
    # position of each step in execution order: units by queue order, a group's steps in order
    pos = step_rank.astype(np.int64) * n + (np.arange(n) - unit)

    # every access as (lo, hi, step, is_write)
    af = sch["acc_first"]
    S = np.repeat(np.arange(n), np.diff(af))
    L, H, Wr = sch["acc_lo"], sch["acc_hi"], sch["acc_write"].astype(bool)
    assert len(S) == len(L) and (H > L).all()
    o = np.argsort(L, kind="stable")
    L, H, S, Wr = L[o], H[o], S[o], Wr[o]
    step_edge = np.zeros(n, dtype=np.int64)
    for t, s in enumerate(tasks["step"]):
        k = -int(tasks["chunk"][t]) if tasks["chunk"][t] < 0 else 1
        step_edge[s:s + k] = tasks["edge"][t]
    # all overlapping pairs of two steps, one of them writing, by a sweep over start points
    pairs = cross = 0
    for i in range(len(L)):
        j = i + 1 + np.nonzero(L[i + 1:np.searchsorted(L, H[i], "left")] < H[i])[0]
        j = j[(S[j] != S[i]) & (Wr[j] | Wr[i])]
        for k in j:
            a, b = int(S[i]), int(S[k])
            if pos[a] > pos[b]:
                a, b = b, a
            if unit[a] == unit[b]:
                continue  # one warp runs a group's steps in order
            ra, rb = int(step_rank[a]), int(step_rank[b])
            assert (anc[rb] >> ra) & 1, f"steps {a} and {b} touch the same elements unordered"
            pairs += 1
            cross += int(step_edge[a] != step_edge[b])
    return len(order), max(depth) + 1, pairs, cross


@pytest.mark.parametrize("queue_order", [0, 1, 2])
@pytest.mark.parametrize("group_rows", [0, -1, 1 << 20])
def test_tree_schedule_is_race_free(qtlib, group_rows, queue_order):
    n = 16
    edges = random_regular_graph(n, 3, 31)
    plan = _plan(n, edges, 2, group_rows=group_rows, queue_order=queue_order)
    from paper_2106_15740_gb300 import binding as qb
    try:
        units, depth, pairs, cross = check_schedule(*_schedule(plan))
    finally:
        qb.qt_plan_free(plan)
    assert cross == 0  # one slot per network: nothing shared between edges
    if group_rows <= 0:  # (with every step grouped, each network is a single task)
        assert pairs > 0 and depth < units


@pytest.mark.parametrize("queue_order", [0, 1, 2])
def test_tree_schedule_with_shared_slots_is_race_free(qtlib, queue_order):
    """A workspace cap puts several networks on one slot: a network's first
    steps then reuse the arena of the network before it."""
    from paper_2106_15740_gb300 import binding as qb
    n = 16
    edges = random_regular_graph(n, 3, 32)
    full = _plan(n, edges, 3)
    data = _data_bytes(full)
    qb.qt_plan_free(full)
    plan = _plan(n, edges, 3, max_workspace=data // 3, queue_order=queue_order)
    try:
        units, depth, pairs, cross = check_schedule(*_schedule(plan))
    finally:
        qb.qt_plan_free(plan)
    assert cross > 0  # networks of one slot reuse each other's arena
    assert pairs > 0 and depth < units


@pytest.mark.parametrize("queue_order", [0, 1, 2])
def test_chain_schedule_is_one_path_per_slot(qtlib, queue_order):
    from paper_2106_15740_gb300 import binding as qb
    n = 12
    edges = random_regular_graph(n, 3, 33)
    plan = _plan(n, edges, 2, chain=1, group_rows=-1, queue_order=queue_order)
    try:
        sch, tasks = _schedule(plan)
        units, depth, _, _ = check_schedule(sch, tasks)
    finally:
        qb.qt_plan_free(plan)
    assert (sch["dep_count"] <= 1).all()
    # one path per slot: each network's steps all lie on its slot's path
    per_edge = np.bincount(tasks["edge"][tasks["chunk"] <= 0])
    assert depth >= per_edge.max()


def test_tree_schedule_of_searched_orders_is_race_free(qtlib):
    """Randomised greedy orders and complex128 (other arena sizes)."""
    from paper_2106_15740_gb300 import binding as qb
    n = 20
    edges = random_regular_graph(n, 3, 34)
    plan = _plan(n, edges, 2, B=3, order_trials=8, dtype=qb.QT_C128)
    try:
        units, depth, pairs, _ = check_schedule(*_schedule(plan))
    finally:
        qb.qt_plan_free(plan)
    assert pairs > 0 and depth < units


@pytest.mark.parametrize("dtype", ["c64", "c64x2"])
@pytest.mark.parametrize("queue_order", [0, 1, 2])
@pytest.mark.parametrize("checkpoint", [False, True])
def test_gradient_schedule_is_race_free(qtlib, checkpoint, queue_order, dtype):
    """The adjoint sweep reads the forward intermediates again, writes output
    adjoints (zeroed first where it accumulates them) and reuses the arena;
    with checkpointing it also re-runs forward steps.  Several networks share
    a slot under a workspace cap.  Float pairs (FP64 adjoints, 16-byte
    elements) take the same schedule rules."""
    from paper_2106_15740_gb300 import binding as qb
    n = 14
    edges = random_regular_graph(n, 3, 35)
    es = 8 if dtype == "c64" else 16

    def grad_plan(cap, ckpt):
        opt = qb.qt_plan_options_default()
        opt.batch = 2
        opt.dtype = qb.QT_C64 if dtype == "c64" else qb.QT_C64X2
        opt.mode = qb.QT_MODE_PERSISTENT
        opt.gradient = 1
        opt.max_workspace = cap
        opt.checkpoint_bytes = ckpt
        opt.queue_order = queue_order
        return qb.qt_plan_create(n, edges, 2, opt)

    full = grad_plan(0, 0)
    data = _data_bytes(full, es)
    qb.qt_plan_free(full)
    plan = grad_plan(data * 2 // 3, (4096 if checkpoint else 0) * es // 8)
    try:
        units, depth, pairs, cross = check_schedule(*_schedule(plan))
    finally:
        qb.qt_plan_free(plan)
    assert pairs > 0 and cross > 0 and depth < units


def test_schedule_rejects_per_bucket_plans(qtlib):
    from paper_2106_15740_gb300 import binding as qb
    n = 8
    edges = random_regular_graph(n, 3, 37)
    opt = qb.qt_plan_options_default()
    opt.batch = 2
    opt.mode = qb.QT_MODE_PER_BUCKET
    plan = qb.qt_plan_create(n, edges, 1, opt)
    try:
        with pytest.raises(qb.QTError):
            qb.qt_plan_schedule(plan)
    finally:
        qb.qt_plan_free(plan)


def test_checker_finds_a_dropped_dependency(qtlib):
    """The check itself: remove the dependencies of one step that reads
    another task's output and the pair is reported unordered."""
    from paper_2106_15740_gb300 import binding as qb
    n = 12
    edges = random_regular_graph(n, 3, 36)
    plan = _plan(n, edges, 2, group_rows=-1)
    try:
        sch, tasks = _schedule(plan)
    finally:
        qb.qt_plan_free(plan)
    check_schedule(sch, tasks)
    # a step that reads an intermediate (it has a read access) and waits for something
    s = next(s for s in range(len(sch["unit"]))
             if sch["dep_count"][s] > 0 and not sch["acc_write"][sch["acc_first"][s]:sch["acc_first"][s + 1]].all())
    bad = dict(sch)
    bad["dep_count"] = sch["dep_count"].copy()
    bad["dep_count"][s] = 0
    with pytest.raises(AssertionError, match="unordered"):
        check_schedule(bad, tasks)


def test_default_grouping_by_batch(qtlib):
    """group_rows = 0: one angle set runs every step as its own task (its
    tiny steps run side by side); larger batches group tiny consecutive
    forward steps."""
    from paper_2106_15740_gb300 import binding as qb
    n = 16
    edges = random_regular_graph(n, 3, 38)
    for B, grouped in ((1, False), (4, True), (64, True)):
        plan = _plan(n, edges, 3, B=B)
        try:
            tasks = qb.qt_plan_tasks(plan)
        finally:
            qb.qt_plan_free(plan)
        assert bool((tasks["chunk"] < 0).any()) == grouped, B


def test_per_width_chunks_schedule_is_race_free(qtlib):
    """Per-width schedule: steps of output rank >= 6 in tasks of 2 tiles,
    rank >= 9 in tasks of 4; every step still completes its own tiles and the
    schedule stays race free."""
    from paper_2106_15740_gb300 import binding as qb
    n = 20
    edges = random_regular_graph(n, 3, 35)
    by_rank = {r: (2 if r < 9 else 4) for r in range(6, 32)}
    base = _plan(n, edges, 3, B=64)
    plan = _plan(n, edges, 3, B=64, by_rank=by_rank)
    try:
        t0, t1 = qb.qt_plan_tasks(base), qb.qt_plan_tasks(plan)
        assert len(t1["step"]) < len(t0["step"])
        units, depth, pairs, _ = check_schedule(*_schedule(plan))
    finally:
        qb.qt_plan_free(plan)
        qb.qt_plan_free(base)
    assert pairs > 0 and depth < units


@pytest.mark.parametrize("field,value", [("chain_steps", 2), ("chain_steps", -1), ("queue_order", 3),
                                         ("queue_order", -1)])
def test_schedule_options_are_validated(qtlib, field, value):
    from paper_2106_15740_gb300 import binding as qb
    opt = qb.qt_plan_options_default()
    assert opt.chain_steps == 0 and opt.queue_order == 2
    opt.batch = 2
    opt.mode = qb.QT_MODE_PERSISTENT
    setattr(opt, field, value)
    with pytest.raises(qb.QTError) as ei:
        qb.qt_plan_create(8, random_regular_graph(8, 3, 39), 1, opt)
    assert ei.value.status == qb.QT_EINVAL


def test_float_pair_gradient_plans_take_at_most_16_angle_sets(qtlib):
    from paper_2106_15740_gb300 import binding as qb
    opt = qb.qt_plan_options_default()
    opt.mode, opt.dtype, opt.gradient, opt.batch = qb.QT_MODE_PERSISTENT, qb.QT_C64X2, 1, 17
    with pytest.raises(qb.QTError) as ei:
        qb.qt_plan_create(8, random_regular_graph(8, 3, 39), 1, opt)
    assert ei.value.status == qb.QT_EINVAL
    for B in (1, 2, 16):
        opt.batch = B
        qb.qt_plan_free(qb.qt_plan_create(8, random_regular_graph(8, 3, 39), 1, opt))
    opt.gradient, opt.batch = 0, 17
    qb.qt_plan_free(qb.qt_plan_create(8, random_regular_graph(8, 3, 39), 1, opt))


def test_per_width_chunks_are_validated(qtlib):
    from paper_2106_15740_gb300 import binding as qb
    opt = qb.qt_plan_options_default()
    assert list(opt.chunk_tiles_by_rank) == [0] * 32
    opt.mode = qb.QT_MODE_PERSISTENT
    opt.chunk_tiles_by_rank[5] = -1
    with pytest.raises(qb.QTError) as ei:
        qb.qt_plan_create(8, random_regular_graph(8, 3, 39), 1, opt)
    assert ei.value.status == qb.QT_EINVAL


def test_sliced_gradient_schedule_is_race_free(qtlib):
    """Sliced networks (2^s restricted copies per edge, some falling apart
    into components whose scalar adjoints read the other scalars) under the
    dependency lists."""
    from paper_2106_15740_gb300 import binding as qb
    n = 12
    edges = random_regular_graph(n, 3, 40)
    opt = qb.qt_plan_options_default()
    opt.batch = 2
    opt.dtype = qb.QT_C64
    opt.mode = qb.QT_MODE_PERSISTENT
    opt.gradient = 1
    opt.max_width = 5
    opt.slice = 1
    plan = qb.qt_plan_create(n, edges, 2, opt)
    try:
        assert qb.qt_plan_edge_slices(plan, len(edges)).max() > 0
        units, depth, pairs, _ = check_schedule(*_schedule(plan))
    finally:
        qb.qt_plan_free(plan)
    assert pairs > 0 and depth < units


def test_amplitude_schedule_is_race_free(qtlib):
    from paper_2106_15740_gb300 import binding as qb
    n = 14
    edges = random_regular_graph(n, 3, 41)
    bits = np.random.default_rng(5).integers(0, 2, size=(6, n))
    opt = qb.qt_plan_options_default()
    opt.batch = 1
    opt.dtype = qb.QT_C128
    opt.mode = qb.QT_MODE_PERSISTENT
    plan = qb.qt_amplitude_plan_create(n, edges, 2, bits, opt)
    try:
        units, depth, pairs, _ = check_schedule(*_schedule(plan))
    finally:
        qb.qt_plan_free(plan)
    assert pairs > 0 and depth < units


def test_schedule_sweep_of_random_configurations(qtlib):
    """A seeded sweep over small plans: graph size and seed, depth, batch,
    dtype (complex64, complex128, float pairs), energy or gradient,
    checkpoint budget, workspace cap, queue order, chained or
    dependency-list schedule and grouping.  Every schedule must pass the
    check."""
    from paper_2106_15740_gb300 import binding as qb
    rng = np.random.default_rng(2106)
    checked = 0
    for trial in range(64):
        n = int(rng.choice([6, 8, 10, 12]))
        p = int(rng.integers(1, 3 if n > 8 else 4))
        edges = random_regular_graph(n, 3, int(rng.integers(0, 1000)))
        opt = qb.qt_plan_options_default()
        opt.batch = int(rng.choice([1, 2, 3, 8, 64]))
        opt.dtype = int(rng.choice([qb.QT_C64, qb.QT_C128, qb.QT_C64X2]))
        opt.mode = qb.QT_MODE_PERSISTENT
        opt.gradient = int(rng.integers(0, 2))
        if opt.gradient and opt.dtype == qb.QT_C64X2 and opt.batch > 16:
            opt.batch = 8  # float-pair gradients take at most 16 angle sets
        opt.queue_order = int(rng.integers(0, 3))
        opt.chain_steps = int(rng.random() < 0.2)
        opt.group_rows = int(rng.choice([0, -1, 64]))
        if opt.gradient and rng.integers(0, 2):
            opt.checkpoint_bytes = int(rng.choice([1 << 10, 1 << 14]))
        plan = qb.qt_plan_create(n, edges, p, opt)
        data = _data_bytes(plan, 8 if opt.dtype == qb.QT_C64 else 16)
        qb.qt_plan_free(plan)
        if rng.integers(0, 2):  # several networks per workspace slot, if the cap allows
            opt.max_workspace = data * 3 // 4
            try:
                plan = qb.qt_plan_create(n, edges, p, opt)
            except qb.QTError:
                opt.max_workspace = 0
                plan = qb.qt_plan_create(n, edges, p, opt)
        else:
            plan = qb.qt_plan_create(n, edges, p, opt)
        try:
            check_schedule(*_schedule(plan))
            checked += 1
        finally:
            qb.qt_plan_free(plan)
    assert checked == 64


def test_schedule_stats_module(qtlib):
    from paper_2106_15740_gb300.schedule import compare
    n = 16
    edges = random_regular_graph(n, 3, 42)
    res = compare(n, edges, 3, batch=4, group_rows=-1)
    tree, chain = res["dependency lists"], res["chained"]
    assert tree["units"] == chain["units"] > 0
    assert chain["max_deps"] == 1 and tree["max_deps"] >= 1
    assert tree["longest_path"] < chain["longest_path"]


def test_trace_stats_on_a_synthetic_trace():
    """Two warps, bins of 10 ns: warp 0 waits 0-10 and works 10-40; warp 1
    works 0-20, then waits 20-25 and works 25-40."""
    from paper_2106_15740_gb300.schedule import trace_stats
    tr = np.array([[0, 10, 40, 0], [0, 0, 20, 1], [20, 25, 40, 1]], dtype=np.uint64) + np.array(
        [100, 100, 100, 0], dtype=np.uint64)
    st = trace_stats(tr, n_warps=2, bin_ns=10, busy_frac=1.0)
    assert st["span_ns"] == 40
    assert st["work_frac"] == pytest.approx((30 + 20 + 15) / 80)
    assert st["wait_frac"] == pytest.approx((10 + 5) / 80)
    assert st["idle_frac"] == pytest.approx(0.0)
    # bins [0,10) .. [40,50): warp 0 works in bins 1-3; warp 1 in bins 0-1, half of 2, and 3
    np.testing.assert_allclose(st["working_warps"], [1.0, 2.0, 1.5, 2.0, 0.0])
    np.testing.assert_allclose(st["waiting_warps"], [1.0, 0.0, 0.5, 0.0, 0.0])
    assert st["full_after_ns"] == 20 and st["tail_ns"] == 0


@pytest.mark.parametrize("gradient", [0, 1])
def test_bytes_by_rank_sums_to_the_plan_bytes(qtlib, gradient):
    """The per-step element counts of the schedule, split at any rank, add
    up to the plan's algorithmic bytes: exactly for forward plans; gradient
    plans add their zeroing steps and scalar adjoints."""
    from paper_2106_15740_gb300 import binding as qb
    from paper_2106_15740_gb300.schedule import bytes_by_rank
    n = 14
    edges = random_regular_graph(n, 3, 43)
    opt = qb.qt_plan_options_default()
    opt.batch = 4
    opt.dtype = qb.QT_C64
    opt.mode = qb.QT_MODE_PERSISTENT
    opt.gradient = gradient
    plan = qb.qt_plan_create(n, edges, 3, opt)
    try:
        total = qb.qt_plan_stats(plan)["alg_bytes"]
        sums = [sum(bytes_by_rank(plan, 4, 8, t).values()) for t in (2, 6, 10, 40)]
        assert max(sums) == pytest.approx(min(sums), rel=1e-12)  # the split does not lose bytes
        if gradient:  # plus the zeroing steps and scalar adjoints, not in the algorithmic count
            assert total <= sums[0] <= 1.1 * total
        else:
            assert sums[0] == pytest.approx(total, rel=1e-12)
        assert bytes_by_rank(plan, 4, 8, 40)["rank>=40"] == 0.0
    finally:
        qb.qt_plan_free(plan)
