"""Seeded randomised greedy elimination orders, in plain Python (test
infrastructure only; nothing in the product path imports this module).

§Results orders its networks with a randomised greedy heuristic that it
names (``rgreedy``) and parametrises (repeats, temperature) without stating
the algorithm.  The library fixes one variant, and this module restates that
specification on its own, so that the orders the benchmark runs with can be
checked element by element:

* Interaction graph: one vertex per variable, an edge between the two
  variables of every rank-2 tensor (the clique of each tensor).
* Score of an alive variable v at a step: f(v) = fill(v) + deg(v) / (n + 1),
  fill = pairs of neighbours of v that are not adjacent, deg = neighbours,
  n = number of variables of the network.  The degree term only breaks ties
  between equal fill-ins (it is below 1).
* Draw: v is taken with probability w(v) / sum w, w(v) = exp(-(f(v) - f_min)
  / tau) (zero once the exponent passes 40).  The uniform number of step s of
  trial t comes from the counter-based generator SplitMix64 (Steele, Lea and
  Flood, 2014): r = M(M(M(seed) xor t) xor s), where M is one SplitMix64
  output for a given state; u = (r >> 11) / 2^53 * sum w, and the variables
  are walked in ascending id, taking the first whose weight exceeds what is
  left of u (the last positive-weight variable if rounding leaves u over).
* Eliminating v records deg(v) (the rank of its bucket result), joins its
  neighbours pairwise and removes v.  Width = largest recorded degree;
  cost = sum over steps of 2^(deg + 1), the elements of each bucket's
  variable set U (|U| = deg + 1), the paper's 2^C measure summed over
  buckets.
* Search: start from greedy min-fill (``lightcone.min_fill_order``); trial
  t = 0, 1, ... replaces the kept order when its width is at most
  max(w_cap, kept width) and its cost is smaller (or equal with a smaller
  width).  The library plans edge e of a graph with seed
  (order_seed << 32) xor e and w_cap = 0, so a kept order is never wider than
  min-fill.

Parity status: SplitMix64 is pinned by its published output sequence, the
draw by the sampling law it must follow, and the search by brute force over
all orders of small networks (``tests/test_oracle_orders.py``).
"""
from __future__ import annotations

import math

import numpy as np

from . import lightcone as lc

_MASK64 = (1 << 64) - 1
_GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(state: int) -> int:
    """The SplitMix64 output for generator state ``state``: advance the state
    by the golden-ratio increment, then the mix with shifts 30, 27, 31 and
    the two published odd multipliers."""
    z = (state + _GOLDEN_GAMMA) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def step_bits(seed: int, trial: int, step: int) -> int:
    """64 random bits of step ``step`` of trial ``trial`` (counter-based)."""
    return splitmix64(splitmix64(splitmix64(seed & _MASK64) ^ (trial & _MASK64)) ^ (step & _MASK64))


def _scores(A, alive, n):
    """f(v) = fill(v) + deg(v) / (n + 1) for every variable (dense 0/1
    adjacency A; the entries of eliminated variables are meaningless)."""
    deg = A.sum(axis=1)
    linked_pairs = (A * (A @ A)).sum(axis=1) / 2.0   # edges among the neighbours
    fill = deg * (deg - 1.0) / 2.0 - linked_pairs
    return fill, deg


def random_greedy(n_vars, tensor_vars, tau, seed, trial):
    """One randomised greedy elimination: (order, width, cost)."""
    A = lc.interaction_graph(n_vars, tensor_vars)
    alive = np.ones(n_vars, dtype=bool)
    order, width, cost = [], 0, 0.0
    for step in range(n_vars):
        fill, deg = _scores(A, alive, n_vars)
        live = [int(v) for v in np.flatnonzero(alive)]
        f = {v: float(fill[v]) + float(deg[v]) / (n_vars + 1) for v in live}
        f_min = min(f.values())
        weight = {}
        total = 0.0
        for v in live:                      # ascending id; a plain running sum
            x = (f[v] - f_min) / tau
            weight[v] = 0.0 if x > 40.0 else math.exp(-x)
            total += weight[v]
        u = float(step_bits(seed, trial, step) >> 11) * 2.0 ** -53 * total
        pick = None
        for v in live:
            if weight[v] <= 0.0:
                continue
            pick = v
            if u < weight[v]:
                break
            u -= weight[v]
        v = pick
        nbrs = np.flatnonzero(A[v])
        width = max(width, len(nbrs))
        cost += float(2 ** (len(nbrs) + 1))
        A[np.ix_(nbrs, nbrs)] = 1.0
        A[nbrs, nbrs] = 0.0
        A[v, :] = 0.0
        A[:, v] = 0.0
        alive[v] = False
        order.append(v)
    return order, width, cost


def order_cost(n_vars, tensor_vars, order):
    """(width, cost) of eliminating the variables in ``order``."""
    adj = [set() for _ in range(n_vars)]
    for vs in tensor_vars:
        for a in vs:
            adj[a].update(x for x in vs if x != a)
    width, cost = 0, 0.0
    for v in order:
        nb = adj[v]
        width = max(width, len(nb))
        cost += float(2 ** (len(nb) + 1))
        for a in nb:
            adj[a].discard(v)
            adj[a].update(nb - {a})
        adj[v] = set()
    return width, cost


def search_order(n_vars, tensor_vars, trials, tau=1.0, seed=0, w_cap=0):
    """Min-fill, then ``trials`` randomised greedy orders; the kept order as
    stated in the module docstring.  Returns (order, width, cost)."""
    order, width = lc.min_fill_order(n_vars, tensor_vars)
    _, cost = order_cost(n_vars, tensor_vars, order)
    for t in range(trials):
        o, w, c = random_greedy(n_vars, tensor_vars, tau, seed, t)
        if w <= max(w_cap, width) and (c < cost or (c == cost and w < width)):
            order, width, cost = o, w, c
    return order, width, cost


def edge_seed(order_seed: int, edge: int) -> int:
    """The seed the library's plans use for edge ``edge``."""
    return ((order_seed & 0xFFFFFFFF) << 32) ^ (edge & 0xFFFFFFFF)
