"""Representation cost study: how much the ZZ and diagonal-gate simplifications
save (§Results, Fig. diag_costs, Fig. diag_costs_vs_n, Tables 1 and 2).

For one amplitude <0...0|psi> of the MaxCut QAOA circuit on seeded random
3-regular graphs, every one of the four gate representations
(``qt_representation``: default, diagonal, ZZ, ZZ + diagonal) is ordered by
the library's greedy min-fill, or the best of min-fill and seeded randomised
greedy orders, and reports its contraction width C and cost sum_b 2^{|U_b|}
(the paper's FLOP measure, about 2^C, up to a constant).  Host only: no
device memory.  Memory limits follow §Results: a tensor of width C takes
16 * 2^C bytes in complex128; a laptop has 4 GB, a supercomputer 800 TB.

    python -m paper_2106_15740_gb300.cost_study            # the tables below
"""
from __future__ import annotations

import math

import numpy as np

from . import binding as qb

REPRESENTATIONS = {"default": qb.QT_REP_DEFAULT, "diagonal": qb.QT_REP_DIAGONAL, "zz": qb.QT_REP_ZZ,
                   "zz+diagonal": qb.QT_REP_ZZ_DIAGONAL}
LAPTOP_BYTES = 4e9
SUPERCOMPUTER_BYTES = 800e12


def _graph(n, seed):
    from workloads import random_regular_graph  # seeded inputs shared with the tests and the bench
    return random_regular_graph(n, 3, seed)


def costs(n, p, seeds=range(5), order_trials=10):
    """{representation: array [len(seeds), 3] of (n_vars, width, log2 cost)}."""
    out = {}
    for name, rep in REPRESENTATIONS.items():
        rows = [qb.qt_representation_cost(n, _graph(n, s), p, rep, order_trials, s) for s in seeds]
        out[name] = np.array(rows, dtype=np.float64)
    return out


def fits(width, budget_bytes, bytes_per_element=16):
    """Largest tensor of the contraction fits the memory budget."""
    return bytes_per_element * math.ldexp(1.0, int(width)) <= budget_bytes


def cost_vs_p(n=40, ps=range(1, 6), seeds=range(5), order_trials=10):
    """Rows (p, representation, mean log2 cost, std, min width, max width)."""
    rows = []
    for p in ps:
        c = costs(n, p, seeds, order_trials)
        for name, a in c.items():
            rows.append((p, name, a[:, 2].mean(), a[:, 2].std(), int(a[:, 1].min()), int(a[:, 1].max())))
    return rows


def cost_vs_n(p=1, ns=(20, 40, 60, 80, 100, 120, 160, 200, 240), seeds=range(5), order_trials=10):
    rows = []
    for n in ns:
        c = costs(n, p, seeds, order_trials)
        for name, a in c.items():
            rows.append((n, name, a[:, 2].mean(), a[:, 2].std(), int(a[:, 1].min()), int(a[:, 1].max())))
    return rows


def max_p(budget_bytes, n=40, p_max=8, seeds=range(5), order_trials=10):
    """Table 1: per representation the largest p whose median width fits."""
    out = {}
    for name, rep in REPRESENTATIONS.items():
        best = 0
        for p in range(1, p_max + 1):
            w = np.median([qb.qt_representation_cost(n, _graph(n, s), p, rep, order_trials, s)[1] for s in seeds])
            if not fits(w, budget_bytes):
                break
            best = p
        out[name] = best
    return out


def max_n(budget_bytes, p=1, ns=range(20, 401, 4), seeds=range(3), order_trials=10):
    """Table 2: per representation the largest N (of `ns`) whose median width fits."""
    out = {}
    for name, rep in REPRESENTATIONS.items():
        best = 0
        for n in ns:
            w = np.median([qb.qt_representation_cost(n, _graph(n, s), p, rep, order_trials, s)[1] for s in seeds])
            if not fits(w, budget_bytes):
                break
            best = n
        out[name] = best
    return out


def main():
    print("log2 cost (mean over 5 graphs) and width range, N = 40, one amplitude")
    for p, name, m, sd, w0, w1 in cost_vs_p():
        print(f"  p={p} {name:12s} log2 cost {m:6.1f} +- {sd:4.1f}  width {w0}-{w1}")
    print("log2 cost vs N, p = 1")
    for n, name, m, sd, w0, w1 in cost_vs_n():
        print(f"  N={n:3d} {name:12s} log2 cost {m:6.1f} +- {sd:4.1f}  width {w0}-{w1}")
    for label, budget in (("laptop 4 GB", LAPTOP_BYTES), ("supercomputer 800 TB", SUPERCOMPUTER_BYTES)):
        print(f"{label}: max p at N = 40 {max_p(budget)}; max N at p = 1 {max_n(budget)}")


if __name__ == "__main__":
    main()
