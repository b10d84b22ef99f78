"""Reference gradients of the QAOA energy (test infrastructure only).

* ``fd_gradient``: central finite differences of any energy function,
  dE/dtheta ~ (E(theta + h) - E(theta - h)) / (2 h).
* ``param_shift_gradient``: the parameter-shift rule on the state vector.
  Every gate of the ansatz is exp(-i theta P) with P^2 = I (P = Z_j Z_k for
  the ZZ phase, P = X for the mixer), so the expectation is
  a + b cos(2 theta) + c sin(2 theta) in the angle of any single gate and its
  derivative is exactly f(theta + pi/4) - f(theta - pi/4).  A layer angle is
  shared by all gates of its layer, so dE/dgamma_q sums the shifts of every
  ZZ gate of layer q and dE/dbeta_q those of every mixer of layer q.
"""
from __future__ import annotations

import numpy as np

from . import statevector as sv


def fd_gradient(energy_fn, gamma, beta, h=1e-5):
    """Returns (dE/dgamma[p], dE/dbeta[p]) for energy_fn(gamma, beta) -> float."""
    gamma = np.asarray(gamma, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    p = gamma.size
    dg, db = np.zeros(p), np.zeros(p)
    for q in range(p):
        e = np.zeros(p)
        e[q] = h
        dg[q] = (energy_fn(gamma + e, beta) - energy_fn(gamma - e, beta)) / (2 * h)
        db[q] = (energy_fn(gamma, beta + e) - energy_fn(gamma, beta - e)) / (2 * h)
    return dg, db


def _energy_pergate(n, edges, g_eq, b_jq, cut):
    psi = sv.qaoa_state_pergate(n, edges, g_eq, b_jq)
    return float(np.dot(np.abs(psi) ** 2, cut))


def param_shift_gradient(n, edges, gamma, beta):
    """Exact (dE/dgamma[p], dE/dbeta[p]) from per-gate shifts of +-pi/4."""
    gamma = np.asarray(gamma, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    p, m = gamma.size, len(edges)
    g_eq = np.repeat(gamma[:, None], m, axis=1)
    b_jq = np.repeat(beta[:, None], n, axis=1)
    cut = sv.cut_values(n, edges)
    s = np.pi / 4
    dg, db = np.zeros(p), np.zeros(p)
    for q in range(p):
        for e in range(m):
            gp, gm = g_eq.copy(), g_eq.copy()
            gp[q, e] += s
            gm[q, e] -= s
            dg[q] += _energy_pergate(n, edges, gp, b_jq, cut) - _energy_pergate(n, edges, gm, b_jq, cut)
        for j in range(n):
            bp, bm = b_jq.copy(), b_jq.copy()
            bp[q, j] += s
            bm[q, j] -= s
            db[q] += _energy_pergate(n, edges, g_eq, bp, cut) - _energy_pergate(n, edges, g_eq, bm, cut)
    return dg, db
