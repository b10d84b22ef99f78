"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers: random d-regular graphs (the paper's
workloads are random 3-regular MaxCut graphs, §Results) and QAOA angle sets
gamma, beta ~ U(0, pi).  It contains none of the method's arithmetic, so both
the CPU oracle and the GPU path may import it.

Generator: numpy's PCG64 (``numpy.random.default_rng(seed)``).  Graphs use the
configuration (pairing) model with rejection of self-loops and multi-edges.
Edges are returned with u < v, sorted lexicographically.
"""
from __future__ import annotations

import numpy as np

# Named workloads: (n_vertices, degree, p, graph seed).  Parameter seeds are
# 1000 + graph seed.  Sizes follow the random 3-regular graphs of §Results.
WORKLOADS = {
    "n16_p1": dict(n=16, d=3, p=1, seed=0),
    "n100_p3": dict(n=100, d=3, p=3, seed=1),
    "n100_p4": dict(n=100, d=3, p=4, seed=2),
    "n60_p4": dict(n=60, d=3, p=4, seed=3),
    "n244_p5": dict(n=244, d=3, p=5, seed=4),
}


def random_regular_graph(n: int, d: int, seed: int, max_tries: int = 100000):
    """Return an (m, 2) int32 array of edges of a uniform-ish random d-regular
    graph on n vertices, drawn by the pairing model with rejection."""
    if n * d % 2:
        raise ValueError("n*d must be even")
    if d >= n:
        raise ValueError("degree must be < n")
    rng = np.random.default_rng(seed)
    stubs = np.repeat(np.arange(n, dtype=np.int64), d)
    for _ in range(max_tries):
        perm = rng.permutation(stubs)
        a, b = perm[0::2], perm[1::2]
        if np.any(a == b):
            continue
        u, v = np.minimum(a, b), np.maximum(a, b)
        key = u * n + v
        if np.unique(key).size != key.size:
            continue
        order = np.lexsort((v, u))
        return np.stack([u[order], v[order]], axis=1).astype(np.int32)
    raise RuntimeError("pairing model did not produce a simple graph")


def random_angles(batch: int, p: int, seed: int):
    """gamma, beta of shape (batch, p), i.i.d. U(0, pi), float64."""
    rng = np.random.default_rng(seed)
    gamma = rng.uniform(0.0, np.pi, size=(batch, p))
    beta = rng.uniform(0.0, np.pi, size=(batch, p))
    return gamma, beta


def erdos_renyi_graph(n: int, prob: float, seed: int):
    """Edges of a G(n, prob) graph (u < v, sorted); used for non-regular cases."""
    rng = np.random.default_rng(seed)
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < prob]
    return np.asarray(edges, dtype=np.int32).reshape(-1, 2)


def complete_graph(n: int):
    return np.asarray([(u, v) for u in range(n) for v in range(u + 1, n)], dtype=np.int32)


def workload(name: str, batch: int = 1):
    """(n, edges, p, gamma[batch, p], beta[batch, p]) for a named workload."""
    w = WORKLOADS[name]
    edges = random_regular_graph(w["n"], w["d"], w["seed"])
    gamma, beta = random_angles(batch, w["p"], 1000 + w["seed"])
    return w["n"], edges, w["p"], gamma, beta
