"""Per-edge lightcone tensor network, min-fill order and naive bucket
elimination, in FP64 (test infrastructure only).

Network (§QAOA algorithm lightcone paragraph; §Tensor network approach;
§Diagonal gate simplification):

* Reverse lightcone of edge (j,k): R_p = {j,k}, R_{q-1} = R_q u N(R_q).
  Layer q keeps the mixers on R_q and the ZZ gates on edges with an endpoint
  in R_q; every other gate cancels against its conjugate.  Qubits of R_0
  start in |+>.
* Every index has dimension 2.  A qubit u with m_u = #{q : u in R_q} mixers
  has ket variables v_u^0..v_u^m and bra variables w_u^0..w_u^{m-1}; its top
  ket and bra variable are one variable (the trace closes there).
* Diagonal gates create no variable (eq. (example)): the ZZ gate of layer q
  is the 2-index tensor [[rho, conj(rho)], [conj(rho), rho]] with
  rho = exp(-i gamma_q) on the current variables of its two qubits, and the
  observable Z is the vector [1, -1] on the top variable.  Mixers (the only
  non-diagonal gates, eq. (zz_gates_circ)) are 2x2 tensors
  [[cos b, -i sin b], [-i sin b, cos b]] from the old to a new variable.
* The bra half holds the elementwise complex conjugate of every ket tensor.

Canonical variable ids: qubits of R_0 in ascending order; for each qubit
v^0, v^1, ..., v^m, then w^{m-1}, ..., w^0.

Order (§Tensor network contraction, Dechter's bucket elimination): greedy
min-fill on the interaction graph (a clique on each tensor's variables):
repeatedly eliminate the variable with the smallest (fill-in, degree, id),
where fill-in counts the missing edges among its neighbours.  The width is the
largest degree met at elimination, i.e. the rank of the largest bucket result.

Contraction: for each variable j in order, multiply every tensor that holds j
and sum over j (§Tensor network contraction).  ``feynman_sum`` evaluates
eq. (tn) literally as a sum over all 2^q assignments.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Network:
    var_names: list = field(default_factory=list)   # (qubit, 'v'|'w', level)
    tensors: list = field(default_factory=list)     # (vars tuple, ndarray)
    tags: list = field(default_factory=list)        # (kind, layer, side)

    @property
    def n_vars(self):
        return len(self.var_names)


def _neighbours(n, edges):
    nb = [set() for _ in range(n)]
    for a, b in edges:
        nb[int(a)].add(int(b))
        nb[int(b)].add(int(a))
    return nb


def reverse_lightcone(n, edges, p, edge_index):
    """Return [R_0, ..., R_p] as sets of qubits."""
    nb = _neighbours(n, edges)
    j, k = (int(x) for x in edges[edge_index])
    R = [None] * (p + 1)
    R[p] = {j, k}
    for q in range(p, 0, -1):
        grown = set(R[q])
        for u in R[q]:
            grown |= nb[u]
        R[q - 1] = grown
    return R


def zz_tensor(gamma):
    """exp(-i gamma z_a z_b) as a 2x2 tensor over the two qubits' bits."""
    same, diff = np.exp(-1j * gamma), np.exp(1j * gamma)
    return np.array([[same, diff], [diff, same]], dtype=np.complex128)


def mixer_tensor(beta):
    """<new| exp(-i beta X) |old> as a 2x2 tensor [new, old]."""
    c, s = np.cos(beta), -1j * np.sin(beta)
    return np.array([[c, s], [s, c]], dtype=np.complex128)


def build_lightcone(n, edges, p, gamma, beta, edge_index) -> Network:
    """The reverse-lightcone network whose full contraction is <Z_j Z_k>."""
    edges = np.asarray(edges)
    gamma = np.asarray(gamma, dtype=np.float64).reshape(p)
    beta = np.asarray(beta, dtype=np.float64).reshape(p)
    R = reverse_lightcone(n, edges, p, edge_index)
    qubits = sorted(R[0])
    m = {u: sum(1 for q in range(1, p + 1) if u in R[q]) for u in qubits}

    net = Network()
    ket, bra = {}, {}
    for u in qubits:
        for lvl in range(m[u] + 1):
            ket[(u, lvl)] = net.n_vars
            net.var_names.append((u, "v", lvl))
        bra[(u, m[u])] = ket[(u, m[u])]
        for lvl in range(m[u] - 1, -1, -1):
            bra[(u, lvl)] = net.n_vars
            net.var_names.append((u, "w", lvl))

    def add(vs, val, tag):
        net.tensors.append((tuple(vs), val))
        net.tags.append(tag)

    plus = np.array([1.0, 1.0], dtype=np.complex128) / np.sqrt(2.0)
    for u in qubits:
        add([ket[(u, 0)]], plus, ("leaf", 0, "ket"))
        add([bra[(u, 0)]], plus.conj(), ("leaf", 0, "bra"))
    for q in range(1, p + 1):
        zz = zz_tensor(gamma[q - 1])
        for a, b in edges:
            a, b = int(a), int(b)
            if a in R[q] or b in R[q]:
                add([ket[(a, q - 1)], ket[(b, q - 1)]], zz, ("zz", q, "ket"))
                add([bra[(a, q - 1)], bra[(b, q - 1)]], zz.conj(), ("zz", q, "bra"))
        mx = mixer_tensor(beta[q - 1])
        for u in sorted(R[q]):
            add([ket[(u, q)], ket[(u, q - 1)]], mx, ("mix", q, "ket"))
            add([bra[(u, q)], bra[(u, q - 1)]], mx.conj(), ("mix", q, "bra"))
    zobs = np.array([1.0, -1.0], dtype=np.complex128)
    j, k = (int(x) for x in edges[edge_index])
    add([ket[(j, m[j])]], zobs, ("obs", p, "ket"))
    add([ket[(k, m[k])]], zobs, ("obs", p, "ket"))
    return net


# ---------------------------------------------------------------------------
# Greedy min-fill elimination order
# ---------------------------------------------------------------------------

def interaction_graph(n_vars, tensor_vars):
    """Adjacency matrix: a clique on the variables of every tensor."""
    A = np.zeros((n_vars, n_vars), dtype=np.float64)
    for vs in tensor_vars:
        for a in vs:
            for b in vs:
                if a != b:
                    A[a, b] = 1.0
    return A


def min_fill_order(n_vars, tensor_vars):
    """Greedy min-fill: returns (order, width).

    fill(v) = deg(v)(deg(v)-1)/2 - #edges among the neighbours of v, where
    twice the edge count among neighbours is (A * (A @ A)).sum(axis=1)[v].
    Ties go to the smaller degree, then to the smaller variable id.
    """
    A = interaction_graph(n_vars, tensor_vars)
    alive = np.ones(n_vars, dtype=bool)
    order, width = [], 0
    for _ in range(n_vars):
        deg = A.sum(axis=1)
        tri2 = (A * (A @ A)).sum(axis=1)
        fill = deg * (deg - 1) / 2 - tri2 / 2
        cand = np.flatnonzero(alive)
        keys = sorted((fill[v], deg[v], v) for v in cand)
        v = int(keys[0][2])
        nbrs = np.flatnonzero(A[v])
        width = max(width, len(nbrs))
        A[np.ix_(nbrs, nbrs)] = 1.0
        A[nbrs, nbrs] = 0.0
        A[v, :] = 0.0
        A[:, v] = 0.0
        alive[v] = False
        order.append(v)
    return order, width


# ---------------------------------------------------------------------------
# Contraction
# ---------------------------------------------------------------------------

def bucket_eliminate(net: Network, order, stats=None):
    """Contract the network variable by variable in ``order``.

    For each variable j: multiply every live tensor that holds j and sum over
    j; the product-sum is one ``numpy.einsum`` call.  Returns the complex
    scalar left when all variables are gone.  If ``stats`` is a list, the
    rank of every bucket result is appended to it.
    """
    live = [(tuple(vs), val) for vs, val in net.tensors]
    for v in order:
        bucket = [t for t in live if v in t[0]]
        live = [t for t in live if v not in t[0]]
        union = sorted({x for vs, _ in bucket for x in vs})
        out_vars = [x for x in union if x != v]
        label = {x: i for i, x in enumerate(union)}
        args = []
        for vs, val in bucket:
            args += [val, [label[x] for x in vs]]
        result = np.einsum(*args, [label[x] for x in out_vars], optimize=False)
        if stats is not None:
            stats.append(len(out_vars))
        live.append((tuple(out_vars), np.asarray(result, dtype=np.complex128)))
    value = np.complex128(1.0)
    for vs, val in live:
        assert len(vs) == 0
        value = value * val[()]
    return complex(value)


def feynman_sum(net: Network):
    """Eq. (tn) literally: sum over all 2^q assignments of the product of
    all tensor entries (one Feynman path per assignment).  q <= 24."""
    q = net.n_vars
    if q > 24:
        raise ValueError("too many variables for brute force")
    idx = np.arange(1 << q, dtype=np.int64)
    path = np.ones(1 << q, dtype=np.complex128)
    for vs, val in net.tensors:
        sub = np.zeros(1 << q, dtype=np.int64)
        for var in vs:
            sub = sub * 2 + ((idx >> var) & 1)
        path *= val.reshape(-1)[sub]
    return complex(path.sum())


def lightcone_zz(n, edges, p, gamma, beta, edge_index):
    """<Z_j Z_k> by bucket elimination in min-fill order; also the width."""
    net = build_lightcone(n, edges, p, gamma, beta, edge_index)
    order, width = min_fill_order(net.n_vars, [vs for vs, _ in net.tensors])
    return bucket_eliminate(net, order), width


def lightcone_energy(n, edges, p, gamma, beta):
    zz = [lightcone_zz(n, edges, p, gamma, beta, e)[0].real for e in range(len(edges))]
    return float(sum(0.5 * (1.0 - z) for z in zz))
