"""The "Default" lightcone network: no diagonal simplification
(test infrastructure only).

§Results compares tensor networks built with and without the diagonal-gate
simplification of §Diagonal gate simplification.  Here every gate is a full
gate tensor that opens new variables: the ZZ phase is the 4-index tensor
D[a', b', a, b] = delta(a', a) delta(b', b) exp(-i gamma z_a z_b) and the
observable is the 2-index tensor Z[j', j] = delta(j', j) (1 - 2 j).  The
lightcone (which gates are kept) is the same as in ``lightcone``.  Its full
contraction equals the simplified network's value -- eq. (example) removes
exactly the delta factors -- while its contraction width is larger.
"""
from __future__ import annotations

import numpy as np

from .lightcone import Network, mixer_tensor, reverse_lightcone


def _zz4(gamma):
    t = np.zeros((2, 2, 2, 2), dtype=np.complex128)
    for a in (0, 1):
        for b in (0, 1):
            s = 1.0 if a == b else -1.0
            t[a, b, a, b] = np.exp(-1j * gamma * s)
    return t


def build_default(n, edges, p, gamma, beta, edge_index) -> Network:
    edges = np.asarray(edges)
    gamma = np.asarray(gamma, dtype=np.float64).reshape(p)
    beta = np.asarray(beta, dtype=np.float64).reshape(p)
    R = reverse_lightcone(n, edges, p, edge_index)
    qubits = sorted(R[0])
    net = Network()

    def new_var(u, side):
        net.var_names.append((u, side, len(net.var_names)))
        return len(net.var_names) - 1

    def side_gates(side):
        """Apply the lightcone circuit on one side; returns each qubit's last variable."""
        conj = (lambda t: t.conj()) if side == "w" else (lambda t: t)
        cur = {}
        plus = np.array([1.0, 1.0], dtype=np.complex128) / np.sqrt(2.0)
        for u in qubits:
            cur[u] = new_var(u, side)
            net.tensors.append(((cur[u],), conj(plus)))
        for q in range(1, p + 1):
            zz = conj(_zz4(gamma[q - 1]))
            for a, b in edges:
                a, b = int(a), int(b)
                if a in R[q] or b in R[q]:
                    na, nb = new_var(a, side), new_var(b, side)
                    net.tensors.append(((na, nb, cur[a], cur[b]), zz))
                    cur[a], cur[b] = na, nb
            mx = conj(mixer_tensor(beta[q - 1]))
            for u in sorted(R[q]):
                nu = new_var(u, side)
                net.tensors.append(((nu, cur[u]), mx))
                cur[u] = nu
        return cur

    ket_top = side_gates("v")
    j, k = (int(x) for x in edges[edge_index])
    zmat = np.diag([1.0, -1.0]).astype(np.complex128)
    for u in (j, k):
        nu = new_var(u, "v")
        net.tensors.append(((nu, ket_top[u]), zmat))
        ket_top[u] = nu
    n_ket = len(net.var_names)
    bra_top = side_gates("w")
    # Close the trace: each qubit's last bra variable is its last ket variable.
    relabel = {bra_top[u]: ket_top[u] for u in qubits}
    tensors = []
    for vs, val in net.tensors:
        tensors.append((tuple(relabel.get(x, x) for x in vs), val))
    keep = [i for i in range(len(net.var_names)) if i not in relabel]
    new_id = {old: i for i, old in enumerate(keep)}
    net.tensors = [(tuple(new_id[x] for x in vs), val) for vs, val in tensors]
    net.var_names = [net.var_names[i] for i in keep]
    assert n_ket <= len(net.var_names)
    return net
