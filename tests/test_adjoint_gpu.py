"""Adjoint gradients on the GPU (hq_adjoint_grad) against the oracle's adjoint
sweep, its parameter-shift rule and FP64 central differences of the oracle's
energies (h = 1e-6).
Bar: relative 1e-4."""
import math

import numpy as np
import pytest

import oracle
from paper_2111_06868_gb300 import circuits as C

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_06868_gb300 import build
    from paper_2111_06868_gb300 import hq as _hq

    build.build()
    _hq.load()
    return _hq


def rel_err(got, want):
    return float(np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-30))


def mixed_circuit(n, layers, seed):
    """Rotations about X, Y, Z and fixed fSim / sqrt(W) gates; one shared parameter."""
    rng = C.SplitMix64(seed)
    gates, p = [], 0
    for _ in range(layers):
        for q in range(n):
            ax = "XYZ"[rng.randint(0, 2)]
            gates.append(C.Gate("R" + ax, (q,), None, ax, p))
            p += 1
        for q in range(0, n - 1, 2):
            gates.append(C.Gate("fSim", (q, q + 1), C.fsim(0.7, 0.3)))
        gates.append(C.Gate("sqrtW", (n - 1,), C.sqrt_w()))
    gates.append(C.Gate("RX", (0,), None, "X", 0))  # parameter 0 used twice
    return C.Circuit(n, gates, p)


def mixed_hamiltonian(n):
    H = [(0.7, ((0, "Y"), (n - 1, "Y"))), (-0.3, ((1, "X"), (2, "Z"))), (0.25, ((n // 2, "Y"),))]
    H += [(0.1 * (q + 1), ((q, "Z"),)) for q in range(n)]
    return H


@pytest.mark.parametrize("dt,tol", [("complex128", 1e-10), ("complex64", 1e-4)])
def test_small_ansatz_matches_oracle(hq, dt, tol):
    circ = C.ansatz(6, 2)
    H = C.ansatz_hamiltonian(6)
    th = C.ansatz_params(circ.n_params, 3, seed=5)
    e, g = hq.hq_adjoint_grad(circ, H, th, dtype=dt)
    for b in range(3):
        e_o, g_o = oracle.adjoint_grad(circ, H, th[b])
        assert abs(e[b] - e_o) <= tol * max(1, abs(e_o))
        assert rel_err(g[b], g_o) <= tol
        assert rel_err(g[b], oracle.param_shift_grad(circ, H, th[b])) <= tol


@pytest.mark.parametrize("dt,tol", [("complex128", 1e-10), ("complex64", 1e-4)])
@pytest.mark.parametrize("tokens", [None, "+-01+-01+"])
def test_mixed_gates_and_y_terms(hq, dt, tol, tokens):
    n = 9
    circ = mixed_circuit(n, 3, seed=2)
    H = mixed_hamiltonian(n)
    th = np.array([[2 * math.pi * ((7 * i + 3 * b) % 11) / 11 for i in range(circ.n_params)] for b in range(2)])
    e, g = hq.hq_adjoint_grad(circ, H, th, dtype=dt, tokens=tokens)
    for b in range(2):
        e_o, g_o = oracle.adjoint_grad(circ, H, th[b], tokens=tokens)
        assert abs(e[b] - e_o) <= tol * max(1, abs(e_o))
        assert rel_err(g[b], g_o) <= tol


def diagonal_mix_circuit(n, n_gates, seed):
    """Rotations about X, Y, Z, dense one-qubit unitaries, CZ and CPhase on
    random pairs (diagonal two-qubit gates whose second qubit lands inside and
    outside the register positions of a run) and a few fSim gates."""
    rng = C.SplitMix64(seed)
    gates, p = [], 0
    for _ in range(n_gates):
        kind = rng.randint(0, 9)
        q = rng.randint(0, n - 1)
        q2 = (q + 1 + rng.randint(0, n - 2)) % n
        if kind <= 3:
            ax = "XYZ"[rng.randint(0, 2)]
            gates.append(C.Gate("R" + ax, (q,), None, ax, p))
            p += 1
        elif kind <= 5:
            gates.append(C.Gate("U", (q,), C.random_unitary(1, rng)))
        elif kind == 6:
            gates.append(C.Gate("CZ", (q, q2), C.cz()))
        elif kind <= 8:
            gates.append(C.Gate("CP", (q, q2), C.cphase(0.3 + rng.uniform())))
        else:
            gates.append(C.Gate("fSim", (q, q2), C.fsim(0.4, 0.9)))
    return C.Circuit(n, gates, p)


@pytest.mark.parametrize("n,seed", [(5, 1), (13, 3), (14, 4)])
def test_register_runs_against_oracle(hq, n, seed):
    """complex64 passes carry runs of sweeps through registers: every mix of
    context bits (inside or outside a run's register positions), elementwise
    diagonal sweeps and dense two-qubit gates between runs against the
    oracle's adjoint."""
    circ = diagonal_mix_circuit(n, 160, seed)
    H = mixed_hamiltonian(n)
    th = np.array([[2 * math.pi * ((5 * i + 7 * b + seed) % 13) / 13 for i in range(circ.n_params)]
                   for b in range(3)])
    e, g = hq.hq_adjoint_grad(circ, H, th, dtype="complex64")
    for b in range(3):
        e_o, g_o = oracle.adjoint_grad(circ, H, th[b])
        assert abs(e[b] - e_o) <= 1e-4 * max(1, abs(e_o))
        assert rel_err(g[b], g_o) <= 1e-4


@pytest.mark.parametrize("checkpoints", [1, 3, 7])
def test_checkpoints_do_not_change_result(hq, checkpoints):
    circ = C.ansatz(8, 3)
    H = C.ansatz_hamiltonian(8)
    th = C.ansatz_params(circ.n_params, 2, seed=9)
    e0, g0 = hq.hq_adjoint_grad(circ, H, th, dtype="complex128")
    e1, g1 = hq.hq_adjoint_grad(circ, H, th, dtype="complex128", checkpoints=checkpoints)
    assert np.max(np.abs(e1 - e0)) <= 1e-12
    assert np.max(np.abs(g1 - g0)) <= 1e-11


@pytest.mark.slow
def test_config_n20_batch64_sampled(hq):
    """n = 20, 8 layers RY RZ + CZ ladder, 320 angles, batch 64: eight sampled
    parameter sets against the oracle's adjoint sweep, and 20 sampled angles
    against FP64 central differences of the oracle's own energies (h = 1e-6)."""
    circ = C.ansatz(20, 8)
    H = C.ansatz_hamiltonian(20)
    th = C.ansatz_params(circ.n_params, 64, seed=0)
    sets = (0, 9, 18, 27, 36, 45, 54, 63)
    ref = {b: oracle.adjoint_grad(circ, H, th[b]) for b in sets}
    grads = {}
    for dt in ("complex64", "complex128"):
        e, g = hq.hq_adjoint_grad(circ, H, th, dtype=dt, checkpoints=4)
        assert e.shape == (64,) and g.shape == (64, 320)
        for b in sets:
            e_o, g_o = ref[b]
            assert abs(e[b] - e_o) <= 1e-4 * max(1, abs(e_o))
            assert rel_err(g[b], g_o) <= 1e-4, (dt, b)
        grads[dt] = g
    h = 1e-6
    b = 18
    angles = list(range(0, 320, 17)) + [319]
    assert len(angles) >= 16
    for p in angles:
        tp, tm = th[b].copy(), th[b].copy()
        tp[p] += h
        tm[p] -= h
        fd = (oracle.energy(circ, H, tp) - oracle.energy(circ, H, tm)) / (2 * h)
        for dt, g in grads.items():
            assert abs(g[b, p] - fd) <= 1e-4 * max(abs(fd), 1e-2 * np.max(np.abs(g[b]))), (dt, p, g[b, p], fd)


def test_autograd_function(hq):
    from paper_2111_06868_gb300.autograd import energy

    circ = C.ansatz(5, 2)
    H = C.ansatz_hamiltonian(5)
    th = torch.tensor(C.ansatz_params(circ.n_params, 2, seed=1), dtype=torch.float64, requires_grad=True)
    e = energy(th, circ, H, dtype="complex128")
    w = torch.tensor([0.5, -2.0], dtype=torch.float64)
    (e * w).sum().backward()
    for b in range(2):
        e_o, g_o = oracle.adjoint_grad(circ, H, th[b].detach().numpy())
        assert abs(e[b].item() - e_o) < 1e-10
        np.testing.assert_allclose(th.grad[b].numpy(), w[b].item() * g_o, atol=1e-10)


def test_adjoint_argument_errors(hq):
    circ = C.ansatz(4, 1)
    H = C.ansatz_hamiltonian(4)
    th = np.zeros((1, circ.n_params))
    bad = C.Circuit(4, circ.gates + [C.Gate("RY", (0,), None, "Y", 99)], circ.n_params)
    with pytest.raises(hq.HQError, match="ARG"):
        hq.hq_adjoint_grad(bad, H, th, dtype="complex128")
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(hq.HQError, match="CAPACITY"):
        hq.hq_adjoint_grad(circ, H, th, dtype="complex128", workspace=small)
