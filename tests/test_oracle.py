"""Pins of the CPU oracle against things other than itself (no GPU).

Each test names what fixes the expected value: the paper's Fig. 1 circuit
(tests/golden), the published p=1 closed form, scipy's matrix exponential,
brute force over bitstrings or assignments, exact invariants, and the
diagonal-simplification identity eq. (example).
"""
import itertools
import json
from pathlib import Path

import numpy as np
import pytest
import scipy.linalg

from oracle import closed_form as cf
from oracle import default_net as dn
from oracle import gradients as gr
from oracle import lightcone as lc
from oracle import statevector as sv
from workloads import complete_graph, erdos_renyi_graph, random_angles, random_regular_graph

GOLDEN = Path(__file__).resolve().parent / "golden"

X = np.array([[0, 1], [1, 0]], dtype=complex)
Z = np.diag([1.0, -1.0]).astype(complex)
H = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)


def _op1(n, q, m):
    """Full 2^n matrix of a one-qubit gate on qubit q (qubit q = bit q)."""
    out = np.array([[1.0 + 0j]])
    for j in range(n - 1, -1, -1):
        out = np.kron(out, m if j == q else np.eye(2))
    return out


def _cnot(n, c, t):
    dim = 1 << n
    M = np.zeros((dim, dim), dtype=complex)
    for x in range(dim):
        y = x ^ (1 << t) if (x >> c) & 1 else x
        M[y, x] = 1
    return M


def _zz_full(n, j, k):
    return _op1(n, j, Z) @ _op1(n, k, Z)


# --------------------------------------------------------------- Fig. 1 ---

def _fig1_state(gamma, beta):
    spec = json.loads((GOLDEN / "fig1_k4_circuit.json").read_text())
    n = spec["n_qubits"]
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1.0

    def apply(op, g, b):
        name = op[0]
        if name == "H":
            return _op1(n, op[1], H)
        if name == "CNOT":
            return _cnot(n, op[1], op[2])
        if name == "ZPOW2G":
            return _op1(n, op[1], np.diag([1.0, np.exp(2j * g)]))
        if name == "ZPOW2B":
            return _op1(n, op[1], np.diag([1.0, np.exp(2j * b)]))
        raise ValueError(name)

    for op in spec["prepare"]:
        psi = apply(op, 0, 0) @ psi
    for g, b in zip(gamma, beta):
        for op in spec["layer"]:
            psi = apply(op, g, b) @ psi
    return n, spec["graph_edges"], psi


@pytest.mark.parametrize("p", [1, 2])
def test_fig1_circuit_fixes_the_convention(p):
    """The paper's Fig. 1 gate sequence (textbook H, CNOT, Z^t) gives the same
    <Z_j Z_k> as the oracle's exp(-i g ZZ), exp(-i b X) ansatz."""
    rng = np.random.default_rng(11 + p)
    for _ in range(3):
        g, b = rng.uniform(0, np.pi, p), rng.uniform(0, np.pi, p)
        n, edges, psi = _fig1_state(g, b)
        prob = np.abs(psi) ** 2
        ref = [float(np.real(np.vdot(psi, _zz_full(n, a, c) @ psi))) for a, c in edges]
        got = sv.edge_zz(n, np.array(edges), g, b)
        np.testing.assert_allclose(got, ref, atol=1e-12)
        assert abs(prob.sum() - 1) < 1e-12


def test_gate_tensors_are_the_paper_gates():
    """eq. (zz_gates_circ) and §Diagonal gate simplification: the ZZ tensor is
    the diagonal of exp(-i g ZZ) (the paper's diag(e^{ig}, e^{-ig}, e^{-ig},
    e^{ig}) with g -> -g), i.e. [[rho, conj rho], [conj rho, rho]] with
    rho = e^{-ig}; the mixer is H Z^{2b} H up to the phase e^{ib}."""
    g, b = 0.37, 1.21
    full = scipy.linalg.expm(-1j * g * np.kron(Z, Z))
    np.testing.assert_allclose(np.diag(np.diag(full)), full, atol=1e-14)  # diagonal
    np.testing.assert_allclose(lc.zz_tensor(g).reshape(-1), np.diag(full), atol=1e-14)
    paper = np.array([np.exp(1j * -g), np.exp(-1j * -g), np.exp(-1j * -g), np.exp(1j * -g)])
    np.testing.assert_allclose(lc.zz_tensor(g).reshape(-1), paper, atol=1e-14)
    rho = np.exp(-1j * g)
    np.testing.assert_allclose(lc.zz_tensor(g), [[rho, rho.conjugate()], [rho.conjugate(), rho]], atol=1e-15)
    hzh = H @ np.diag([1, np.exp(2j * b)]) @ H
    np.testing.assert_allclose(hzh, np.exp(1j * b) * lc.mixer_tensor(b), atol=1e-14)
    np.testing.assert_allclose(lc.mixer_tensor(b), scipy.linalg.expm(-1j * b * X), atol=1e-14)
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    lhs = cnot @ np.kron(np.eye(2), np.diag([1, np.exp(2j * g)])) @ cnot
    np.testing.assert_allclose(lhs, np.exp(1j * g) * full, atol=1e-14)


# --------------------------------------------------------- closed form ----

@pytest.mark.parametrize("graph", ["reg3_n12", "k4", "k5", "gnp_n9"])
def test_statevector_matches_p1_closed_form(graph):
    if graph == "reg3_n12":
        n, edges = 12, random_regular_graph(12, 3, 4)
    elif graph == "k4":
        n, edges = 4, complete_graph(4)
    elif graph == "k5":
        n, edges = 5, complete_graph(5)
    else:
        n, edges = 9, erdos_renyi_graph(9, 0.45, 2)
    rng = np.random.default_rng(5)
    for _ in range(3):
        g, b = rng.uniform(0, np.pi), rng.uniform(0, np.pi)
        zz = sv.edge_zz(n, edges, [g], [b])
        ref = [cf.p1_zz(n, edges, e, g, b) for e in range(len(edges))]
        np.testing.assert_allclose(zz, ref, atol=1e-12)


def test_single_edge_closed_form():
    """N = 2: <ZZ> = sin(4b) sin(2g), from 4x4 matrices."""
    for g, b in [(0.3, 0.9), (1.1, 2.5), (2.9, 0.2)]:
        psi = np.full(4, 0.5, dtype=complex)
        psi = scipy.linalg.expm(-1j * g * np.kron(Z, Z)) @ psi
        psi = np.kron(scipy.linalg.expm(-1j * b * X), scipy.linalg.expm(-1j * b * X)) @ psi
        direct = float(np.real(np.vdot(psi, np.kron(Z, Z) @ psi)))
        assert abs(direct - np.sin(4 * b) * np.sin(2 * g)) < 1e-13
        assert abs(sv.edge_zz(2, np.array([[0, 1]]), [g], [b])[0] - direct) < 1e-13
        assert abs(cf.p1_zz(2, np.array([[0, 1]]), 0, g, b) - direct) < 1e-13


@pytest.mark.parametrize("p", [2, 3])
def test_statevector_matches_matrix_exponential(p):
    """Whole-register evolution with scipy.linalg.expm of the cost and mixer
    Hamiltonians (an independent method) on a small graph."""
    n, edges = 5, erdos_renyi_graph(5, 0.6, 1)
    Hc = sum(_zz_full(n, int(a), int(c)) for a, c in edges)
    Hb = sum(_op1(n, j, X) for j in range(n))
    rng = np.random.default_rng(p)
    g, b = rng.uniform(0, np.pi, p), rng.uniform(0, np.pi, p)
    psi = np.full(1 << n, 2 ** (-n / 2), dtype=complex)
    for q in range(p):
        psi = scipy.linalg.expm(-1j * b[q] * Hb) @ (scipy.linalg.expm(-1j * g[q] * Hc) @ psi)
    np.testing.assert_allclose(sv.qaoa_state(n, edges, g, b), psi, atol=1e-12)


# ---------------------------------------------------------- invariants ----

def test_energy_invariants():
    n, edges = 10, random_regular_graph(10, 3, 7)
    m = len(edges)
    rng = np.random.default_rng(3)
    g, b = rng.uniform(0, np.pi, 3), rng.uniform(0, np.pi, 3)
    # gamma = 0: the state stays |+>, every <ZZ> = 0, E = |E|/2
    assert abs(sv.energy(n, edges, np.zeros(3), b) - m / 2) < 1e-12
    # every beta in {0, pi/2}: <ZZ> = 0
    for bb in (np.zeros(3), np.full(3, np.pi / 2)):
        np.testing.assert_allclose(sv.edge_zz(n, edges, g, bb), 0, atol=1e-12)
    E = sv.energy(n, edges, g, b)
    assert abs(sv.energy(n, edges, -g, -b) - E) < 1e-12                 # time reversal
    assert abs(sv.energy(n, edges, g + np.pi, b) - E) < 1e-12           # gamma period pi
    assert abs(sv.energy(n, edges, g, b + np.pi / 2) - E) < 1e-12       # beta period pi/2
    cut = sv.cut_values(n, edges)
    assert 0 <= E <= cut.max() + 1e-12                                   # 0 <= E <= maxcut
    np.testing.assert_allclose(sv.energy(n, edges, g, b), 0.5 * (m - sv.edge_zz(n, edges, g, b).sum()), atol=1e-12)


# ----------------------------------------------------- lightcone network --

@pytest.mark.parametrize("n,p,seed", [(8, 1, 0), (10, 2, 1), (12, 2, 2), (14, 3, 3), (12, 3, 4)])
def test_lightcone_network_matches_statevector(n, p, seed):
    edges = random_regular_graph(n, 3, seed)
    g, b = random_angles(1, p, 100 + seed)
    zz = sv.edge_zz(n, edges, g[0], b[0])
    for e in range(len(edges)):
        val, _ = lc.lightcone_zz(n, edges, p, g[0], b[0], e)
        assert abs(val.real - zz[e]) < 1e-12
        assert abs(val.imag) < 1e-12


def test_lightcone_on_nonregular_graph():
    n, edges = 9, erdos_renyi_graph(9, 0.4, 5)
    g, b = random_angles(1, 2, 9)
    zz = sv.edge_zz(n, edges, g[0], b[0])
    for e in range(len(edges)):
        assert abs(lc.lightcone_zz(n, edges, 2, g[0], b[0], e)[0] - zz[e]) < 1e-12


@pytest.mark.parametrize("n,p,edge", [(6, 1, 0), (8, 1, 3), (2, 2, 0), (4, 2, 1)])
def test_bucket_elimination_equals_feynman_sum(n, p, edge):
    edges = complete_graph(n) if n <= 4 else random_regular_graph(n, 3, n)
    g, b = random_angles(1, p, 40 + n)
    net = lc.build_lightcone(n, edges, p, g[0], b[0], edge)
    assert net.n_vars <= 24
    order, _ = lc.min_fill_order(net.n_vars, [vs for vs, _ in net.tensors])
    brute = lc.feynman_sum(net)
    assert abs(lc.bucket_eliminate(net, order) - brute) < 1e-12
    # any other order gives the same value
    rev = list(reversed(order))
    assert abs(lc.bucket_eliminate(net, rev) - brute) < 1e-12


def test_diagonal_simplification_is_exact_and_narrower():
    """eq. (example): the network with full 4-index ZZ tensors has the same
    value and a larger contraction width (§Results, "Default" vs "Diagonal")."""
    n, p = 12, 2
    edges = random_regular_graph(n, 3, 8)
    g, b = random_angles(1, p, 8)
    for e in (0, 5, 11):
        diag = lc.build_lightcone(n, edges, p, g[0], b[0], e)
        full = dn.build_default(n, edges, p, g[0], b[0], e)
        assert full.n_vars > diag.n_vars
        od, wd = lc.min_fill_order(diag.n_vars, [vs for vs, _ in diag.tensors])
        of, wf = lc.min_fill_order(full.n_vars, [vs for vs, _ in full.tensors])
        assert abs(lc.bucket_eliminate(full, of) - lc.bucket_eliminate(diag, od)) < 1e-12
        assert wf > wd


def test_tree_like_lightcone_variable_count():
    """Without cycles in the lightcone, |R_q| = 2(2^{p-q+1} - 1) and a qubit with
    m mixers has 2m + 1 variables, so n_vars = sum over R_0 of (2 m_u + 1)."""
    n, p = 200, 2
    edges = random_regular_graph(n, 3, 21)
    checked = 0
    for e in range(len(edges)):
        R = lc.reverse_lightcone(n, edges, p, e)
        if len(R[0]) != 2 * (2 ** (p + 1) - 1):
            continue
        assert [len(R[q]) for q in range(p + 1)] == [2 * (2 ** (p - q + 1) - 1) for q in range(p + 1)]
        net = lc.build_lightcone(n, edges, p, [0.1] * p, [0.2] * p, e)
        expect = sum(2 * sum(1 for q in range(1, p + 1) if u in R[q]) + 1 for u in R[0])
        assert net.n_vars == expect == 2 * 5 + 4 * 3 + 8 * 1
        checked += 1
    assert checked > 100


# -------------------------------------------------------------- ordering --

def _set_min_fill(n_vars, tensor_vars):
    """Min-fill by its definition on adjacency sets (slow, tiny inputs)."""
    adj = {v: set() for v in range(n_vars)}
    for vs in tensor_vars:
        for a in vs:
            adj[a] |= set(vs) - {a}
    order, width = [], 0
    while adj:
        def key(v):
            nb = sorted(adj[v])
            fill = sum(1 for a, c in itertools.combinations(nb, 2) if c not in adj[a])
            return (fill, len(nb), v)
        v = min(adj, key=key)
        nb = adj.pop(v)
        width = max(width, len(nb))
        for a in nb:
            adj[a] |= nb - {a}
            adj[a].discard(v)
        order.append(v)
    return order, width


def test_min_fill_hand_example():
    """Hand-worked: a 4-cycle 0-1-2-3-0 plus a pendant 4 on 0.
    Step 1: 4 has degree 1 and no fill -> eliminate 4.
    Step 2: every cycle vertex has fill 1 and degree 2 -> smallest id, 0;
    fill edge 1-3.  Step 3: 1, 2, 3 form a triangle (fill 0, degree 2) -> 1.
    Then 2 (fill 0, degree 1), then 3.  Width = 2."""
    tv = [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4)]
    order, width = lc.min_fill_order(5, tv)
    assert order == [4, 0, 1, 2, 3] and width == 2


def test_min_fill_matches_set_definition_and_bounds_treewidth():
    rng = np.random.default_rng(0)
    for trial in range(30):
        nv = int(rng.integers(4, 9))
        tv = [tuple(sorted(rng.choice(nv, size=int(rng.integers(1, 4)), replace=False))) for _ in range(nv + 2)]
        tv += [(v,) for v in range(nv)]
        order, width = lc.min_fill_order(nv, tv)
        assert (order, width) == _set_min_fill(nv, tv)
        best = min(_width_of(nv, tv, perm) for perm in itertools.permutations(range(nv)))
        assert width >= best


def _width_of(nv, tv, perm):
    adj = {v: set() for v in range(nv)}
    for vs in tv:
        for a in vs:
            adj[a] |= set(vs) - {a}
    w = 0
    for v in perm:
        nb = adj.pop(v)
        w = max(w, len(nb))
        for a in nb:
            adj[a] |= nb - {a}
            adj[a].discard(v)
    return w


def test_width_is_largest_bucket_result():
    n, edges, p = 16, random_regular_graph(16, 3, 0), 2
    g, b = random_angles(1, p, 3)
    for e in range(0, len(edges), 4):
        net = lc.build_lightcone(n, edges, p, g[0], b[0], e)
        order, width = lc.min_fill_order(net.n_vars, [vs for vs, _ in net.tensors])
        ranks = []
        lc.bucket_eliminate(net, order, stats=ranks)
        assert max(ranks) == width


# ------------------------------------------------------------ gradients ---

def test_gradients_fd_vs_parameter_shift_vs_closed_form():
    n, edges = 8, random_regular_graph(8, 3, 2)
    g, b = np.array([0.7]), np.array([0.4])
    ps = gr.param_shift_gradient(n, edges, g, b)
    fd = gr.fd_gradient(lambda gg, bb: sv.energy(n, edges, gg, bb), g, b)
    # analytic derivative of the published closed form
    import sympy
    G, Bt = sympy.symbols("g b")
    expr = 0
    nb = [set() for _ in range(n)]
    for a, c in edges:
        nb[int(a)].add(int(c))
        nb[int(c)].add(int(a))
    for a, c in edges:
        d, e, lam = len(nb[a]) - 1, len(nb[c]) - 1, len(nb[a] & nb[c])
        zz = (sympy.Rational(1, 2) * sympy.sin(4 * Bt) * sympy.sin(2 * G) * (sympy.cos(2 * G) ** d + sympy.cos(2 * G) ** e)
              + sympy.Rational(1, 2) * sympy.sin(2 * Bt) ** 2 * sympy.cos(2 * G) ** (d + e - 2 * lam) * (1 - sympy.cos(4 * G) ** lam))
        expr += (1 - zz) / 2
    an_g = float(sympy.diff(expr, G).subs({G: 0.7, Bt: 0.4}))
    an_b = float(sympy.diff(expr, Bt).subs({G: 0.7, Bt: 0.4}))
    np.testing.assert_allclose([ps[0][0], ps[1][0]], [an_g, an_b], atol=1e-11)
    np.testing.assert_allclose([fd[0][0], fd[1][0]], [an_g, an_b], atol=1e-8)


def test_gradients_fd_vs_parameter_shift_p2():
    n, edges = 8, random_regular_graph(8, 3, 6)
    g, b = random_angles(1, 2, 66)
    ps = gr.param_shift_gradient(n, edges, g[0], b[0])
    fd = gr.fd_gradient(lambda gg, bb: sv.energy(n, edges, gg, bb), g[0], b[0])
    np.testing.assert_allclose(ps[0], fd[0], atol=1e-8)
    np.testing.assert_allclose(ps[1], fd[1], atol=1e-8)
    fd_tn = gr.fd_gradient(lambda gg, bb: lc.lightcone_energy(n, edges, 2, gg, bb), g[0], b[0])
    np.testing.assert_allclose(fd_tn[0], ps[0], atol=1e-8)
    np.testing.assert_allclose(fd_tn[1], ps[1], atol=1e-8)


# --------------------------------------------------------------- planted --

def test_planted_mistakes_are_caught():
    """Plant plausible oracle mistakes (on the CPU) and check a pin fails."""
    n, edges = 8, random_regular_graph(8, 3, 1)
    g, b = 0.61, 0.33
    ref = [cf.p1_zz(n, edges, e, g, b) for e in range(len(edges))]
    # wrong sign of gamma in the ZZ tensor
    net = lc.build_lightcone(n, edges, 1, [-g], [b], 0)
    order, _ = lc.min_fill_order(net.n_vars, [vs for vs, _ in net.tensors])
    assert abs(lc.bucket_eliminate(net, order).real - ref[0]) > 1e-3
    # bra half not conjugated
    net = lc.build_lightcone(n, edges, 1, [g], [b], 0)
    net.tensors = [(vs, val if tag[2] == "ket" else val.conj()) for (vs, val), tag in zip(net.tensors, net.tags)]
    assert abs(lc.bucket_eliminate(net, order) - ref[0]) > 1e-3
    # dropped mixer term (-i sin b -> 0)
    net = lc.build_lightcone(n, edges, 1, [g], [b], 0)
    net.tensors = [(vs, np.diag(np.diag(val)) if tag[0] == "mix" else val) for (vs, val), tag in zip(net.tensors, net.tags)]
    assert abs(lc.bucket_eliminate(net, order) - ref[0]) > 1e-3
