"""Dense FP64 state-vector QAOA simulator (test infrastructure only).

Implements the ansatz of §QAOA algorithm, eq. (1)/(2): starting from |+>^n,
layer q multiplies every amplitude by exp(-i gamma_q sum_{(j,k)} z_j z_k)
(z = 1 - 2 x, the eigenvalue of Z on bit x) and then applies
exp(-i beta_q X) to every qubit.  Qubit j is bit j of the basis index.

<Z_j Z_k> = sum_x |psi(x)|^2 z_j z_k and E = sum_x |psi(x)|^2 cut(x), the
MaxCut cost C = 1/2 sum (1 - Z_j Z_k) of §QAOA algorithm.

Also offers per-gate angles (one gamma per (layer, edge), one beta per
(layer, qubit)) for the parameter-shift rule.
"""
from __future__ import annotations

import numpy as np


def _zz_sign(n: int, j: int, k: int) -> np.ndarray:
    """z_j z_k for every basis state (+1 if bits equal, -1 otherwise)."""
    x = np.arange(1 << n, dtype=np.int64)
    return 1.0 - 2.0 * (((x >> j) ^ (x >> k)) & 1)


def _apply_rx(psi: np.ndarray, n: int, j: int, beta: float) -> np.ndarray:
    """Apply exp(-i beta X) on qubit j: [[cos b, -i sin b], [-i sin b, cos b]]."""
    c, s = np.cos(beta), -1j * np.sin(beta)
    v = psi.reshape(1 << (n - j - 1), 2, 1 << j)
    a0, a1 = v[:, 0, :].copy(), v[:, 1, :].copy()
    v[:, 0, :] = c * a0 + s * a1
    v[:, 1, :] = s * a0 + c * a1
    return psi


def qaoa_state_pergate(n, edges, gamma_eq, beta_jq):
    """State for per-gate angles.

    gamma_eq: (p, m) angle of the ZZ gate on edge e in layer q.
    beta_jq:  (p, n) angle of the mixer on qubit j in layer q.
    """
    edges = np.asarray(edges)
    p = gamma_eq.shape[0]
    psi = np.full(1 << n, 2.0 ** (-n / 2), dtype=np.complex128)
    signs = [_zz_sign(n, int(a), int(b)) for a, b in edges]
    for q in range(p):
        phase = np.zeros(1 << n)
        for e, sgn in enumerate(signs):
            phase += gamma_eq[q, e] * sgn
        psi *= np.exp(-1j * phase)
        for j in range(n):
            psi = _apply_rx(psi, n, j, beta_jq[q, j])
    return psi


def qaoa_state(n, edges, gamma, beta):
    """|gamma beta>_p for layer angles gamma[p], beta[p]."""
    gamma = np.asarray(gamma, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    m = len(edges)
    g = np.repeat(gamma[:, None], m, axis=1)
    b = np.repeat(beta[:, None], n, axis=1)
    return qaoa_state_pergate(n, edges, g, b)


def zz_expectations(psi, n, edges):
    """<Z_j Z_k> for every edge (float64 array; the state is normalised)."""
    prob = np.abs(psi) ** 2
    return np.array([np.dot(prob, _zz_sign(n, int(a), int(b))) for a, b in edges])


def cut_values(n, edges):
    """cut(x) = number of edges with differing endpoint bits, for every x."""
    x = np.arange(1 << n, dtype=np.int64)
    cut = np.zeros(1 << n)
    for a, b in edges:
        cut += ((x >> int(a)) ^ (x >> int(b))) & 1
    return cut


def energy(n, edges, gamma, beta):
    """E = <gamma beta| C |gamma beta>, C the MaxCut cost."""
    psi = qaoa_state(n, edges, gamma, beta)
    return float(np.dot(np.abs(psi) ** 2, cut_values(n, edges)))


def edge_zz(n, edges, gamma, beta):
    """Per-edge <Z_j Z_k> from the full state vector."""
    return zz_expectations(qaoa_state(n, edges, gamma, beta), n, edges)
