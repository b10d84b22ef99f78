"""Pins of the oracle's randomised greedy orders (oracle/orders.py), then
bit-exact parity of the library's searched orders with them (host only).

§Results orders its networks with a randomised greedy heuristic (rgreedy,
repeats and a temperature); the library specifies one variant and the
oracle restates it.  The pins hold the oracle to things other than itself:
the published SplitMix64 output sequence, the sampling law a draw must
follow, and brute force over every order of small networks.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import lightcone as lc
from oracle import orders as od
from workloads import random_angles, random_regular_graph, workload


def test_splitmix64_published_sequence():
    """SplitMix64 from state 0 (Steele, Lea and Flood 2014; the sequence
    quoted with the generator's reference code): the first five outputs."""
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC,
              0x1B39896A51A8749B]
    state = 0
    for want in expect:
        assert od.splitmix64(state) == want
        state = (state + 0x9E3779B97F4A7C15) % (1 << 64)


def _small_graph():
    """A 7-variable interaction structure: a 4-cycle 0-1-2-3 with chord 0-2,
    a path 3-4-5 and a pendant 6 on 5."""
    return 7, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2), (3, 4), (4, 5), (5, 6)]


def _first_step_law(n, tv, tau):
    """Probability of each variable being eliminated first, from the
    definition: weight exp(-(f - f_min)/tau), f = fill + deg/(n+1), with fill
    and degree counted from the edge list by hand."""
    adj = {v: set() for v in range(n)}
    for a, b in tv:
        adj[a].add(b)
        adj[b].add(a)
    f = {}
    for v in range(n):
        nb = sorted(adj[v])
        missing = sum(1 for a, b in itertools.combinations(nb, 2) if b not in adj[a])
        f[v] = missing + len(nb) / (n + 1)
    fmin = min(f.values())
    w = np.array([math.exp(-(f[v] - fmin) / tau) for v in range(n)])
    return w / w.sum()


@pytest.mark.parametrize("tau", [0.5, 2.0])
def test_first_draw_follows_the_sampling_law(tau):
    n, tv = _small_graph()
    law = _first_step_law(n, tv, tau)
    trials = 6000
    counts = np.zeros(n)
    for t in range(trials):
        order, _, _ = od.random_greedy(n, tv, tau, seed=12345, trial=t)
        counts[order[0]] += 1
    freq = counts / trials
    sigma = np.sqrt(law * (1 - law) / trials)
    assert np.all(np.abs(freq - law) <= 5 * sigma + 1e-12), (freq, law)


def test_cold_draws_take_a_minimal_fill_then_degree_variable():
    """tau -> 0: every step eliminates a variable of minimal (fill, degree);
    checked step by step against a set-based recount."""
    n, edges, p = 12, random_regular_graph(12, 3, 1), 2
    g, b = random_angles(1, p, 5)
    net = lc.build_lightcone(n, edges, p, g[0], b[0], 3)
    tv = [vs for vs, _ in net.tensors]
    order, width, cost = od.random_greedy(net.n_vars, tv, 1e-6, seed=7, trial=3)
    adj = {v: set() for v in range(net.n_vars)}
    for vs in tv:
        for a in vs:
            adj[a] |= set(vs) - {a}
    for v in order:
        def key(u):
            nb = sorted(adj[u])
            return (sum(1 for a, c in itertools.combinations(nb, 2) if c not in adj[a]), len(nb))
        assert key(v) == min(key(u) for u in adj)
        nb = adj.pop(v)
        for a in nb:
            adj[a] |= nb - {a}
            adj[a].discard(v)
    assert (width, cost) == od.order_cost(net.n_vars, tv, order)


def test_order_cost_matches_bucket_elimination_ranks():
    """Width and cost of an order against the ranks the oracle's bucket
    elimination reports: cost = sum_b 2^(rank_b + 1)."""
    n, edges, p = 14, random_regular_graph(14, 3, 2), 2
    g, b = random_angles(1, p, 9)
    for e in (0, 7, 13):
        net = lc.build_lightcone(n, edges, p, g[0], b[0], e)
        tv = [vs for vs, _ in net.tensors]
        order, _, _ = od.random_greedy(net.n_vars, tv, 1.0, seed=3, trial=e)
        ranks = []
        lc.bucket_eliminate(net, order, stats=ranks)
        assert od.order_cost(net.n_vars, tv, order) == (max(ranks), float(sum(2 ** (r + 1) for r in ranks)))


def test_search_reaches_the_brute_force_optimum_on_small_networks():
    """With many hot trials the search finds an order of the least cost over
    all n! orders whose width is within min-fill's, and never returns a
    costlier or wider order than min-fill."""
    rng = np.random.default_rng(4)
    for case in range(6):
        n = int(rng.integers(5, 8))
        tv = sorted({tuple(sorted(rng.choice(n, 2, replace=False))) for _ in range(n + 3)})
        tv += [(v,) for v in range(n)]
        mf_order, mf_w = lc.min_fill_order(n, tv)
        _, mf_cost = od.order_cost(n, tv, mf_order)
        best = min(od.order_cost(n, tv, perm)[1] for perm in itertools.permutations(range(n))
                   if od.order_cost(n, tv, perm)[0] <= mf_w)
        order, w, cost = od.search_order(n, tv, trials=600, tau=4.0, seed=case)
        assert sorted(order) == list(range(n))
        assert (w, cost) == od.order_cost(n, tv, order)
        assert w <= mf_w and cost <= mf_cost
        assert cost == best


def test_search_keeps_min_fill_without_trials():
    n, tv = _small_graph()
    order, w, c = od.search_order(n, tv, trials=0)
    assert (order, w) == lc.min_fill_order(n, tv) and (w, c) == od.order_cost(n, tv, order)


# ------------------------------------------------ library parity (host) ---

def _plan(qb, name, trials, edge_range, batch=1):
    n, edges, p, _, _ = workload(name)
    opt = qb.qt_plan_options_default()
    opt.batch = batch
    opt.dtype = qb.QT_C64
    opt.mode = qb.QT_MODE_PERSISTENT
    opt.order_trials = trials
    opt.edge_begin, opt.edge_end = edge_range
    return qb.qt_plan_create(n, edges, p, opt), n, edges, p


@pytest.mark.parametrize("name,trials,edges_sel", [
    ("n100_p3", 100, (0, 41, 77, 149)),
    ("n100_p4", 100, (5, 62, 118)),
    ("n100_p4", 10, (0, 30, 90, 149)),
])
def test_library_searched_orders_match_oracle_bitwise(qtlib, name, trials, edges_sel):
    """The plan's elimination order and width of each sampled edge equal the
    oracle's search with the same seed (order_seed 0, edge index) -- the
    orders and widths the benchmark's plan runs with (100 trials)."""
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, g, b = workload(name)
    for e in edges_sel:
        plan, *_ = _plan(qb, name, trials, (e, e + 1))
        try:
            lib_order = list(qb.qt_plan_edge_order(plan, 0))
            lib_width = int(qb.qt_plan_edge_widths(plan, 1)[0])
        finally:
            qb.qt_plan_free(plan)
        net = lc.build_lightcone(n, edges, p, g[0], b[0], e)
        order, width, _ = od.search_order(net.n_vars, [vs for vs, _ in net.tensors], trials, tau=1.0,
                                          seed=od.edge_seed(0, e))
        assert lib_order == order and lib_width == width


def test_library_min_fill_plan_order_matches_oracle(qtlib):
    from paper_2106_15740_gb300 import binding as qb
    n, edges, p, g, b = workload("n60_p4")
    plan, *_ = _plan(qb, "n60_p4", 0, (10, 14))
    try:
        for k in range(4):
            net = lc.build_lightcone(n, edges, p, g[0], b[0], 10 + k)
            assert list(qb.qt_plan_edge_order(plan, k)) == lc.min_fill_order(net.n_vars,
                                                                              [vs for vs, _ in net.tensors])[0]
        with pytest.raises(qb.QTError):
            qb.qt_plan_edge_order(plan, 4)
    finally:
        qb.qt_plan_free(plan)
