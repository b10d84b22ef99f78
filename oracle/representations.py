"""The four gate representations of the QAOA amplitude network compared in
§Results (test infrastructure only; nothing in the product path imports
this module).

One amplitude <0...0| U(gamma, beta) |+>^n of the full circuit, written as a
tensor network straight from the gate list of Fig. 1: every edge (j, k) of
layer q is CNOT(j -> k), Z^(2 gamma_q) on k, CNOT(j -> k) (eq.
(zz_gates_circ)); every qubit's mixer is H, Z^(2 beta_q), H.  Z^t is
diag(1, e^{i t}), H and CNOT the textbook gates (the reading the Fig. 1
golden file records).  With this reading the circuit is the library's
exp(-i gamma ZZ) / exp(-i beta X) circuit times the global phase
e^{i sum_q (|E| gamma_q + n beta_q)}.

Representations (§Results, Figs. diag_costs and diag_costs_vs_n):

* ``default``  -- every gate is a tensor with a new index on each qubit it
  acts on: CNOT [c', t', c, t], Z [z', z], H [h', h].
* ``diagonal`` -- the same gates; a gate that is diagonal in one of its
  qubits keeps that qubit's index (§Diagonal gate simplification): Z^t is a
  vector on the current index, CNOT is diagonal in its control and becomes
  [c, t', t].
* ``zz``       -- the edge's three gates merged into one ZZ gate
  diag(1, e^{2i g}, e^{2i g}, 1) with new indices on both qubits, and the
  mixer merged into one gate H Z H with a new index.
* ``zz_diagonal`` -- the merged ZZ gate keeps both indices (a 2-index
  diagonal tensor); the mixer as in ``zz``.  This is the library's
  amplitude network.

Each qubit starts in |+> (a vector on its first index) and its last index
is projected on 0, so it is no variable.  Variables are numbered qubit by
qubit in ascending order and, within a qubit, in the order its gates opened
them.  Width and cost come from the oracle's greedy min-fill
(``lightcone.min_fill_order``): width = largest bucket result rank, cost =
sum over buckets of 2^{|U_b|} (``orders.order_cost``), the paper's 2^C
measure summed over buckets.

Parity status: each network is pinned by contracting it to the state
vector's amplitude (``tests/test_oracle_representations.py``).
"""
from __future__ import annotations

import math

import numpy as np

from . import lightcone as lc
from . import orders as od

REPRESENTATIONS = ("default", "diagonal", "zz", "zz_diagonal")

_H = np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128) / math.sqrt(2.0)
_PLUS = np.array([1.0, 1.0], dtype=np.complex128) / math.sqrt(2.0)


def _zpow(t):
    return np.array([1.0, np.exp(1j * t)], dtype=np.complex128)


def _cnot4():
    """CNOT as a tensor [c_out, t_out, c_in, t_in]."""
    T = np.zeros((2, 2, 2, 2), dtype=np.complex128)
    for c in range(2):
        for t in range(2):
            T[c, t ^ c, c, t] = 1.0
    return T


def _cnot3():
    """CNOT with the control index shared: [c, t_out, t_in]."""
    T = np.zeros((2, 2, 2), dtype=np.complex128)
    for c in range(2):
        for t in range(2):
            T[c, t ^ c, t] = 1.0
    return T


def build(n, edges, p, gamma, beta, rep):
    """The amplitude network <0...0|psi> of representation ``rep``
    (a ``lightcone.Network``; tensor values in the Fig. 1 convention)."""
    if rep not in REPRESENTATIONS:
        raise ValueError(rep)
    edges = [(int(a), int(b)) for a, b in np.asarray(edges).reshape(-1, 2)]
    gamma = np.asarray(gamma, dtype=np.float64).reshape(p)
    beta = np.asarray(beta, dtype=np.float64).reshape(p)
    labels = []          # (qubit, serial) of every opened index
    serial = [0] * n
    cur = [None] * n
    raw = []             # (labels tuple, array)

    def fresh(u):
        lab = (u, serial[u])
        serial[u] += 1
        labels.append(lab)
        cur[u] = lab
        return lab

    for u in range(n):
        raw.append(((fresh(u),), _PLUS))
    diag = rep in ("diagonal", "zz_diagonal")
    for q in range(p):
        g2, b2 = 2.0 * gamma[q], 2.0 * beta[q]
        for a, b in edges:
            if rep == "zz_diagonal":
                raw.append(((cur[a], cur[b]), np.array([[1.0, np.exp(1j * g2)], [np.exp(1j * g2), 1.0]])))
            elif rep == "zz":
                a0, b0 = cur[a], cur[b]
                zz = np.array([[1.0, np.exp(1j * g2)], [np.exp(1j * g2), 1.0]])
                T = np.einsum("ab,ac,bd->cdab", zz, np.eye(2), np.eye(2))   # [a', b', a, b]
                raw.append(((fresh(a), fresh(b), a0, b0), T))
            else:
                for half in range(2):
                    a0, b0 = cur[a], cur[b]
                    if diag:
                        raw.append(((a0, fresh(b), b0), _cnot3()))
                    else:
                        raw.append(((fresh(a), fresh(b), a0, b0), _cnot4()))
                    if half == 0:
                        if diag:
                            raw.append(((cur[b],), _zpow(g2)))
                        else:
                            t0 = cur[b]
                            raw.append(((fresh(b), t0), np.diag(_zpow(g2))))
        for u in range(n):
            if rep in ("zz", "zz_diagonal"):
                u0 = cur[u]
                raw.append(((fresh(u), u0), _H @ np.diag(_zpow(b2)) @ _H))
            else:
                u0 = cur[u]
                raw.append(((fresh(u), u0), _H))
                if diag:
                    raw.append(((cur[u],), _zpow(b2)))
                else:
                    u0 = cur[u]
                    raw.append(((fresh(u), u0), np.diag(_zpow(b2))))
                u0 = cur[u]
                raw.append(((fresh(u), u0), _H))
    projected = set(cur)                      # each qubit's last index, fixed to 0
    kept = sorted(lab for lab in labels if lab not in projected)
    vid = {lab: i for i, lab in enumerate(kept)}
    net = lc.Network()
    net.var_names = kept
    for labs, arr in raw:
        arr = np.asarray(arr, dtype=np.complex128)
        index = tuple(0 if lab in projected else slice(None) for lab in labs)
        net.tensors.append((tuple(vid[lab] for lab in labs if lab not in projected), arr[index]))
        net.tags.append((rep,))
    return net


def global_phase(n, n_edges, gamma, beta):
    """Phase of the Fig. 1 circuit relative to the exp(-i gamma ZZ),
    exp(-i beta X) circuit: e^{i sum_q (|E| gamma_q + n beta_q)}."""
    return np.exp(1j * (n_edges * float(np.sum(gamma)) + n * float(np.sum(beta))))


def cost(n, edges, p, rep, trials=0, seed=0):
    """(n_vars, width, log2 cost) of representation ``rep`` under min-fill,
    or under the order search with ``trials`` randomised orders."""
    net = build(n, edges, p, np.zeros(p), np.zeros(p), rep)
    tv = [vs for vs, _ in net.tensors]
    if trials > 0:
        order, width, c = od.search_order(net.n_vars, tv, trials, 1.0, od.edge_seed(seed, 0))
    else:
        order, width = lc.min_fill_order(net.n_vars, tv)
        _, c = od.order_cost(net.n_vars, tv, order)
    return net.n_vars, width, math.log2(c)
