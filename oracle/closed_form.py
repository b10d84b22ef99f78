"""Published p=1 closed form for <Z_j Z_k> (test infrastructure only).

Source: Z. Wang, S. Hadfield, Z. Jiang, E. Rieffel, "Quantum approximate
optimization algorithm for MaxCut: a fermionic view", PRA 97, 022304 (2018),
Theorem 1, which gives <C_uv> for U_C = exp(-i g C), U_B = exp(-i b B).

Restated in this library's convention, where the ZZ gate is
exp(-i gamma Z_j Z_k): since exp(-i g (1 - ZZ)/2) equals exp(+i g/2 ZZ) up to
a phase, g = -2 gamma.  With d = deg(j) - 1, e = deg(k) - 1 and lambda the
number of triangles containing edge (j,k):

  <Z_j Z_k> = 1/2 sin(4 beta) sin(2 gamma) (cos^d(2 gamma) + cos^e(2 gamma))
            + 1/2 sin^2(2 beta) cos^(d+e-2 lambda)(2 gamma) (1 - cos^lambda(4 gamma)).

For a single edge (N=2) this reduces to sin(4 beta) sin(2 gamma).
"""
from __future__ import annotations

import numpy as np


def _neighbours(n, edges):
    nb = [set() for _ in range(n)]
    for a, b in edges:
        nb[int(a)].add(int(b))
        nb[int(b)].add(int(a))
    return nb


def p1_zz(n, edges, edge_index, gamma, beta):
    """<Z_j Z_k> at p=1 for edge ``edge_index`` of the graph."""
    nb = _neighbours(n, edges)
    j, k = (int(x) for x in edges[edge_index])
    d = len(nb[j]) - 1
    e = len(nb[k]) - 1
    lam = len(nb[j] & nb[k])
    c2 = np.cos(2 * gamma)
    term1 = 0.5 * np.sin(4 * beta) * np.sin(2 * gamma) * (c2 ** d + c2 ** e)
    term2 = 0.5 * np.sin(2 * beta) ** 2 * c2 ** (d + e - 2 * lam) * (1 - np.cos(4 * gamma) ** lam)
    return float(term1 + term2)


def p1_energy(n, edges, gamma, beta):
    return float(sum(0.5 * (1 - p1_zz(n, edges, i, gamma, beta)) for i in range(len(edges))))
