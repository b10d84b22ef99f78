"""Single amplitudes <x|psi(gamma, beta)> of the full circuit against the oracle.

References: the oracle's 2^n FP64 state vector (qubit u = bit u of the basis
index) for every bitstring of 10-vertex graphs, its normalisation, the
closed form at gamma = 0 (every mixer leaves |+> invariant up to the phase
exp(-i beta_q), so <x|psi> = exp(-i n sum_q beta_q) / 2^(n/2) for every x),
and, on a 40-vertex p = 2 graph with no state vector, the sliced plan
(2^6 restricted networks per bitstring) against the unsliced one and
complex64 against complex128.
Tolerances: complex128 1e-12 absolute (each amplitude is about 2^-n/2 in
size); complex64 1e-5 relative to the largest amplitude, the relative size of
the complex64 energy tolerance (1e-5 on values of order 1).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import statevector as sv
from workloads import random_angles, random_regular_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(qtlib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return qtlib


def _all_bits(n):
    x = np.arange(1 << n, dtype=np.int64)
    return ((x[:, None] >> np.arange(n)) & 1).astype(np.uint8)


def _amps(plan, g, b):
    amp = plan.amplitudes(torch.tensor(g, device="cuda:0"), torch.tensor(b, device="cuda:0"))
    plan.check()
    a = amp.cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]  # [n_strings, B]


@pytest.mark.parametrize("mode", ["persistent", "per_bucket"])
@pytest.mark.parametrize("dtype", ["c128", "c64", "c64x2"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_every_amplitude_matches_state_vector(mode, dtype, p):
    from paper_2106_15740_gb300.amplitude import AmplitudePlan
    n, B = 10, 2
    edges = random_regular_graph(n, 3, 30 + p)
    g, b = random_angles(B, p, 40 + p)
    bits = _all_bits(n)
    plan = AmplitudePlan(n, edges, p, bits, batch=B, dtype=dtype, mode=mode, device="cuda:0")
    amp = _amps(plan, g, b)
    plan.close()
    for k in range(B):
        ref = sv.qaoa_state(n, edges, g[k], b[k])
        tol = 1e-5 * np.abs(ref).max() if dtype == "c64" else 1e-12
        assert np.abs(amp[:, k] - ref).max() <= tol
        assert abs(np.sum(np.abs(amp[:, k]) ** 2) - 1.0) <= (1e-5 if dtype == "c64" else 1e-10)


def test_gamma_zero_closed_form_on_40_vertices():
    from paper_2106_15740_gb300.amplitude import AmplitudePlan
    n, p, B = 40, 2, 3
    edges = random_regular_graph(n, 3, 50)
    g, b = random_angles(B, p, 51)
    g[:] = 0.0
    bits = np.random.default_rng(52).integers(0, 2, (4, n)).astype(np.uint8)
    plan = AmplitudePlan(n, edges, p, bits, batch=B, dtype="c128", device="cuda:0")
    amp = _amps(plan, g, b)
    plan.close()
    for k in range(B):
        ref = np.exp(-1j * n * b[k].sum()) * 2.0 ** (-n / 2)
        assert np.abs(amp[:, k] - ref).max() <= 1e-12 * 2.0 ** (-n / 2) * 1e3


def test_sliced_and_complex64_agree_with_unsliced_complex128_on_40_vertices_p2():
    from paper_2106_15740_gb300.amplitude import AmplitudePlan
    n, p, B = 40, 2, 2
    edges = random_regular_graph(n, 3, 53)
    g, b = random_angles(B, p, 54)
    bits = np.random.default_rng(55).integers(0, 2, (2, n)).astype(np.uint8)
    full = AmplitudePlan(n, edges, p, bits, batch=B, dtype="c128", order_trials=50, device="cuda:0")
    assert max(full.widths) <= 20 and max(full.slices) == 0
    a0 = _amps(full, g, b)
    full.close()
    sliced = AmplitudePlan(n, edges, p, bits, batch=B, dtype="c128", order_trials=50, max_width=12, slice=True,
                           max_workspace=8 << 30, device="cuda:0")
    assert max(sliced.widths) <= 12 and min(sliced.slices) >= 1
    a1 = _amps(sliced, g, b)
    sliced.close()
    scale = np.abs(a0).max()
    assert np.abs(a1 - a0).max() <= 1e-11 * max(scale, 2.0 ** (-n / 2))
    c64 = AmplitudePlan(n, edges, p, bits, batch=B, dtype="c64", order_trials=50, device="cuda:0")
    a2 = _amps(c64, g, b)
    c64.close()
    assert np.abs(a2 - a0).max() <= 1e-5 * scale


def test_amplitude_and_energy_calls_do_not_mix():
    from paper_2106_15740_gb300 import binding as qb
    from paper_2106_15740_gb300.amplitude import AmplitudePlan
    from paper_2106_15740_gb300.energy import EnergyPlan
    n, p = 10, 1
    edges = random_regular_graph(n, 3, 56)
    amp_plan = AmplitudePlan(n, edges, p, _all_bits(n)[:4], device="cuda:0")
    g = torch.zeros((1, p), dtype=torch.float64, device="cuda:0")
    with pytest.raises(qb.QTError):
        qb.qt_plan_energy(amp_plan.plan, g.data_ptr(), g.data_ptr(), 0, 0, 0, amp_plan.workspace.data_ptr(),
                          amp_plan.ws_bytes, 0)
    amp_plan.close()
    e_plan = EnergyPlan(n, edges, p, device="cuda:0")
    out = torch.empty((len(edges), 1, 2), dtype=torch.float64, device="cuda:0")
    with pytest.raises(qb.QTError):
        qb.qt_plan_amplitudes(e_plan.plan, g.data_ptr(), g.data_ptr(), out.data_ptr(), e_plan.workspace.data_ptr(),
                              e_plan.ws_bytes, 0)
    e_plan.close()
