"""Pins of the oracle's four amplitude-network representations
(oracle/representations.py), then bit-exact parity of the library's
representation cost study (qt_representation_cost) with them.

§Results compares the contraction cost of one amplitude under four gate
representations (default, diagonal, ZZ, ZZ + diagonal).  Each oracle network
is built from the Fig. 1 gate list and pinned by contracting it: all four
must give the state vector's amplitude <0...0|psi> (times the global phase
of the Fig. 1 gates).  The library builds only the interaction structure;
its variable count, min-fill width and log2 cost must equal the oracle's.
"""
import math

import numpy as np
import pytest

from oracle import lightcone as lc
from oracle import representations as rp
from oracle import statevector as sv
from workloads import random_angles, random_regular_graph

REP_ID = {"default": 0, "diagonal": 1, "zz": 2, "zz_diagonal": 3}


@pytest.mark.parametrize("rep", rp.REPRESENTATIONS)
@pytest.mark.parametrize("n,p,seed", [(6, 1, 0), (8, 2, 3), (6, 3, 5)])
def test_network_contracts_to_the_state_vector_amplitude(rep, n, p, seed):
    edges = random_regular_graph(n, 3, seed)
    g, b = random_angles(1, p, 60 + seed)
    net = rp.build(n, edges, p, g[0], b[0], rep)
    order, _ = lc.min_fill_order(net.n_vars, [vs for vs, _ in net.tensors])
    amp = lc.bucket_eliminate(net, order)
    ref = sv.qaoa_state(n, edges, g[0], b[0])[0] * rp.global_phase(n, len(edges), g[0], b[0])
    assert abs(amp - ref) <= 1e-12 * max(1.0, abs(ref)) + 1e-14


def _default_amp(n, edges, p, g, b):
    net = rp.build(n, edges, p, g, b, "default")
    order, _ = lc.min_fill_order(net.n_vars, [vs for vs, _ in net.tensors])
    return lc.bucket_eliminate(net, order)


def test_reversed_cnot_pairs_give_the_same_amplitude():
    """CNOT, Z on the target, CNOT is exp(i g) exp(-i g ZZ), symmetric in its
    two qubits: the pair with control and target exchanged is the same gate."""
    n, p = 6, 2
    edges = random_regular_graph(n, 3, 1)
    g, b = random_angles(1, p, 11)
    ref = sv.qaoa_state(n, edges, g[0], b[0])[0] * rp.global_phase(n, len(edges), g[0], b[0])
    assert abs(_default_amp(n, [(int(v), int(u)) for u, v in edges], p, g[0], b[0]) - ref) < 1e-12


def test_planted_gate_mistakes_change_the_amplitude(monkeypatch):
    """Mistakes planted in the oracle's gates -- CNOT with control and target
    exchanged inside the tensor, Z^t read as diag(1, e^{-it}) -- no longer
    give the state vector's amplitude."""
    n, p = 6, 2
    edges = random_regular_graph(n, 3, 1)
    g, b = random_angles(1, p, 11)
    ref = sv.qaoa_state(n, edges, g[0], b[0])[0] * rp.global_phase(n, len(edges), g[0], b[0])
    assert abs(_default_amp(n, edges, p, g[0], b[0]) - ref) < 1e-12

    def wrong_cnot():
        T = np.zeros((2, 2, 2, 2), dtype=np.complex128)
        for c in range(2):
            for t in range(2):
                T[c ^ t, t, c, t] = 1.0   # the target flips the control
        return T

    with monkeypatch.context() as m:
        m.setattr(rp, "_cnot4", wrong_cnot)
        assert abs(_default_amp(n, edges, p, g[0], b[0]) - ref) > 1e-6
    with monkeypatch.context() as m:
        m.setattr(rp, "_zpow", lambda t: np.array([1.0, np.exp(-1j * t)], dtype=np.complex128))
        assert abs(_default_amp(n, edges, p, g[0], b[0]) - ref) > 1e-6


@pytest.mark.parametrize("n,p", [(8, 1), (10, 3)])
def test_variable_counts(n, p):
    """Opened indices minus the n projected outputs: ZZ + diagonal n p; ZZ
    two more per ZZ gate; diagonal one per CNOT target and per Hadamard;
    default one per gate index."""
    edges = random_regular_graph(n, 3, 2)
    m = len(edges)
    expect = {"zz_diagonal": n * p, "zz": n * p + 2 * m * p, "diagonal": p * (2 * n + 2 * m),
              "default": p * (3 * n + 5 * m)}
    for rep, nv in expect.items():
        assert rp.build(n, edges, p, np.zeros(p), np.zeros(p), rep).n_vars == nv


@pytest.mark.parametrize("n,p,seed", [(10, 1, 0), (10, 3, 1), (16, 2, 2), (20, 1, 3), (20, 3, 4)])
def test_library_cost_study_matches_oracle_bitwise(qtlib, n, p, seed):
    from paper_2106_15740_gb300 import binding as qb
    edges = random_regular_graph(n, 3, seed)
    for rep in rp.REPRESENTATIONS:
        nv, w, lc2 = rp.cost(n, edges, p, rep)
        lnv, lw, llc2 = qb.qt_representation_cost(n, edges, p, REP_ID[rep])
        assert (lnv, lw) == (nv, w)
        assert llc2 == pytest.approx(lc2, abs=1e-12)


def test_library_searched_cost_matches_oracle(qtlib):
    """With randomised orders (seed 3, 8 trials) as well."""
    from paper_2106_15740_gb300 import binding as qb
    n, p = 14, 2
    edges = random_regular_graph(n, 3, 7)
    for rep in ("diagonal", "zz_diagonal"):
        nv, w, lc2 = rp.cost(n, edges, p, rep, trials=8, seed=3)
        lnv, lw, llc2 = qb.qt_representation_cost(n, edges, p, REP_ID[rep], 8, 3)
        assert (lnv, lw) == (nv, w) and math.isclose(llc2, lc2, abs_tol=1e-12)
