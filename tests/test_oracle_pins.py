"""Pins for the CPU oracle: closed forms, brute force, and the paper's printed
examples.  None of these re-types the oracle's own formula; each would fail on a
plausible slip in it (wrong bit order, transposed matrix, dropped term, sign).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2111_06868_gb300 import circuits as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# brute force: the full 2^n x 2^n matrix of one gate, straight from the
# definition U[y, x] = M[r(y), r(x)] if y, x agree off the targets, else 0.
# --------------------------------------------------------------------------
def full_unitary(n, qubits, M):
    dim = 1 << n
    U = np.zeros((dim, dim), np.complex128)
    bits = [n - 1 - q for q in qubits]
    tmask = sum(1 << b for b in bits)
    k = len(qubits)

    def local(x):
        return sum(((x >> bits[j]) & 1) << (k - 1 - j) for j in range(k))

    for y in range(dim):
        for x in range(dim):
            if (y & ~tmask) == (x & ~tmask):
                U[y, x] = M[local(y), local(x)]
    return U


def brute_force_state(circuit, psi0):
    psi = psi0.copy()
    for g in circuit.gates:
        psi = full_unitary(circuit.n, g.qubits, g.matrix) @ psi
    return psi


def kron_state(tokens):
    vec = {
        "0": np.array([1, 0], np.complex128),
        "1": np.array([0, 1], np.complex128),
        "+": np.array([1, 1], np.complex128) / math.sqrt(2),
        "-": np.array([1, -1], np.complex128) / math.sqrt(2),
    }
    out = np.array([1], np.complex128)
    for t in tokens:  # np.kron(a, b): a is the more significant factor
        out = np.kron(out, vec[t])
    return out


def test_grover_printout_pins_qubit_order():
    """Sec. 2.2: inverting the phase of |00> on qubits 1, 2 of the uniform
    3-qubit state negates entries 000 and 100 (printed amplitudes)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "grover_sec2_2.txt")) if not l.startswith("#")]
    psi = oracle.state_init(3, "+++")
    flip = np.diag([-1, 1, 1, 1]).astype(np.complex128)  # I - 2|00><00|
    oracle.apply_gate(psi, 3, [1, 2], flip)
    for bits, val in rows:
        i = int(bits, 2)
        assert abs(psi[i].imag) < 1e-15
        assert f"{psi[i].real:+g}" == val


@pytest.mark.parametrize("tokens", ["0", "1", "+", "-", "01", "+-", "10+-", "-+10-", "0+1-0+1-"])
def test_state_init_matches_kron(tokens):
    psi = oracle.state_init(len(tokens), tokens)
    np.testing.assert_allclose(psi, kron_state(tokens), atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
def test_ghz_closed_form(n):
    psi = oracle.simulate(C.ghz_circuit(n))
    expect = np.zeros(1 << n, np.complex128)
    expect[0] = expect[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(psi, expect, atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_qft_of_basis_state(n):
    N = 1 << n
    for x in sorted({0, 1, N - 1, (5 * N) // 7, N // 2}):
        circ = C.Circuit(n, C.basis_prep(n, x).gates + C.qft_circuit(n).gates)
        psi = oracle.simulate(circ)
        y = np.arange(N)
        expect = np.exp(2j * math.pi * x * y / N) / math.sqrt(N)
        np.testing.assert_allclose(psi, expect, atol=1e-13)


def test_sqrt_gates_on_basis_states():
    """Non-symmetric 1q gates pin row/column order: sqrt(Y)|0> = |+>,
    sqrt(Y)|1> = -|->; sqrt(X)|0> = (|0> - i|1>)/sqrt 2."""
    s = 1 / math.sqrt(2)
    psi = oracle.state_init(1, "0")
    oracle.apply_gate(psi, 1, [0], C.sqrt_y())
    np.testing.assert_allclose(psi, [s, s], atol=1e-15)
    psi = oracle.state_init(1, "1")
    oracle.apply_gate(psi, 1, [0], C.sqrt_y())
    np.testing.assert_allclose(psi, [-s, s], atol=1e-15)
    psi = oracle.state_init(1, "0")
    oracle.apply_gate(psi, 1, [0], C.sqrt_x())
    np.testing.assert_allclose(psi, [s, -1j * s], atol=1e-15)


def test_cnot_control_is_first_qubit():
    """CNOT(control=qubits[0]) on |10> gives |11>; on |01> it does nothing."""
    psi = oracle.state_init(2, "10")
    oracle.apply_gate(psi, 2, [0, 1], C.cnot())
    assert abs(psi[3] - 1) < 1e-15
    psi = oracle.state_init(2, "01")
    oracle.apply_gate(psi, 2, [0, 1], C.cnot())
    assert abs(psi[1] - 1) < 1e-15
    # reversed qubit list: control is qubit 1
    psi = oracle.state_init(2, "01")
    oracle.apply_gate(psi, 2, [1, 0], C.cnot())
    assert abs(psi[3] - 1) < 1e-15


@pytest.mark.parametrize("n,kmax,seed", [(1, 1, 0), (2, 2, 1), (3, 3, 2), (5, 3, 3), (6, 6, 4), (7, 4, 5), (8, 3, 6)])
def test_brute_force_full_unitary(n, kmax, seed):
    circ = C.random_dense_circuit(n, 12, seed, kmax)
    psi0 = kron_state(("+-01" * 4)[:n])
    got = oracle.apply_circuit(psi0.copy(), circ)
    want = brute_force_state(circ, psi0)
    np.testing.assert_allclose(got, want, atol=1e-13)


def test_norm_preserved_and_inverse_returns_to_zero():
    circ = C.config_small(seed=3)
    psi = oracle.simulate(circ)
    assert abs(oracle.norm2(psi) - 1) < 1e-13
    oracle.apply_circuit(psi, circ.inverse())
    expect = np.zeros_like(psi)
    expect[0] = 1
    np.testing.assert_allclose(psi, expect, atol=1e-13)


def test_norm2_closed_form():
    psi = np.arange(8, dtype=np.float64) + 1j * np.ones(8)
    assert oracle.norm2(psi.astype(np.complex128)) == pytest.approx(sum(i * i + 1 for i in range(8)), rel=1e-15)


# --------------------------------------------------------------------------
# expectation values
# --------------------------------------------------------------------------
def pauli_matrix(n, term):
    out = np.array([[1]], np.complex128)
    s = C.pauli_string(n, term)
    for p in s:
        out = np.kron(out, C.PAULI[p])
    return out


def test_expectation_single_qubit_closed_forms():
    assert oracle.expectation(oracle.state_init(1, "0"), [(1.0, ((0, "Z"),))]) == pytest.approx(1)
    assert oracle.expectation(oracle.state_init(1, "1"), [(1.0, ((0, "Z"),))]) == pytest.approx(-1)
    assert oracle.expectation(oracle.state_init(1, "+"), [(1.0, ((0, "X"),))]) == pytest.approx(1)
    assert oracle.expectation(oracle.state_init(1, "-"), [(1.0, ((0, "X"),))]) == pytest.approx(-1)
    psi = oracle.state_init(1, "0")
    oracle.apply_gate(psi, 1, [0], C.rot("X", -math.pi / 2))  # (|0> + i|1>)/sqrt 2
    assert oracle.expectation(psi, [(1.0, ((0, "Y"),))]) == pytest.approx(1, abs=1e-15)
    # RY(pi/2) on qubit j gives <X_j> = 1 (the other qubits stay |0>)
    psi = oracle.state_init(4, "0000")
    oracle.apply_gate(psi, 4, [2], C.rot("Y", math.pi / 2))
    assert oracle.expectation(psi, [(1.0, ((2, "X"),))]) == pytest.approx(1, abs=1e-15)
    assert oracle.expectation(psi, [(1.0, ((1, "X"),))]) == pytest.approx(0, abs=1e-15)
    # ZZ on |01> = -1, Z0 on |01> = +1 (qubit 0 is the MSB)
    psi = oracle.state_init(2, "01")
    assert oracle.expectation(psi, [(1.0, ((0, "Z"), (1, "Z")))]) == pytest.approx(-1)
    assert oracle.expectation(psi, [(1.0, ((1, "Z"),))]) == pytest.approx(-1)
    assert oracle.expectation(psi, [(1.0, ((0, "Z"),))]) == pytest.approx(1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_expectation_brute_force(seed):
    n = 5
    circ = C.random_dense_circuit(n, 10, seed, 3)
    psi = oracle.simulate(circ)
    rng = C.SplitMix64(100 + seed)
    H = []
    for _ in range(6):
        L = rng.randint(1, 3)
        qs = []
        while len(qs) < L:
            q = rng.randint(0, n - 1)
            if q not in qs:
                qs.append(q)
        H.append((rng.uniform() - 0.5, tuple((q, "XYZ"[rng.randint(0, 2)]) for q in qs)))
    want = sum(c * np.vdot(psi, pauli_matrix(n, t) @ psi).real for c, t in H)
    assert oracle.expectation(psi, H) == pytest.approx(want, abs=1e-13)


def test_ansatz_zero_angles_energy():
    """All angles 0: the ansatz leaves |0..0>; E = (n-1) ZZ terms of +1, X terms 0."""
    n = 8
    circ = C.ansatz(n, 2)
    e = oracle.energy(circ, C.ansatz_hamiltonian(n), np.zeros(circ.n_params))
    assert e == pytest.approx(n - 1, abs=1e-13)


# --------------------------------------------------------------------------
# gradients
# --------------------------------------------------------------------------
def test_gradient_single_rotation_closed_form():
    """RY(t)|0> with H = Z: E = cos t, dE/dt = -sin t; RX with H = Y:
    E = -sin t, dE/dt = -cos t."""
    for t in [0.3, 1.7, 4.0]:
        circ = C.Circuit(1, [C.Gate("RY", (0,), None, "Y", 0)], 1)
        e, g = oracle.adjoint_grad(circ, [(1.0, ((0, "Z"),))], [t])
        assert e == pytest.approx(math.cos(t), abs=1e-14)
        assert g[0] == pytest.approx(-math.sin(t), abs=1e-14)
        circ = C.Circuit(1, [C.Gate("RX", (0,), None, "X", 0)], 1)
        e, g = oracle.adjoint_grad(circ, [(1.0, ((0, "Y"),))], [t])
        assert e == pytest.approx(-math.sin(t), abs=1e-14)
        assert g[0] == pytest.approx(-math.cos(t), abs=1e-14)


@pytest.mark.parametrize("n,layers,seed", [(3, 1, 0), (5, 2, 1)])
def test_gradient_adjoint_vs_shift_vs_finite_difference(n, layers, seed):
    circ = C.ansatz(n, layers)
    H = C.ansatz_hamiltonian(n)
    theta = C.ansatz_params(circ.n_params, 1, seed)[0]
    e, g_adj = oracle.adjoint_grad(circ, H, theta)
    assert e == pytest.approx(oracle.energy(circ, H, theta), abs=1e-13)
    g_ps = oracle.param_shift_grad(circ, H, theta)
    h = 1e-6
    g_fd = np.empty_like(g_adj)
    for p in range(circ.n_params):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        g_fd[p] = (oracle.energy(circ, H, tp) - oracle.energy(circ, H, tm)) / (2 * h)
    np.testing.assert_allclose(g_adj, g_ps, atol=1e-12)
    np.testing.assert_allclose(g_adj, g_fd, atol=1e-8)


# --------------------------------------------------------------------------
# sequence matrix (matrix(circuit) of Sec. 3.1)
# --------------------------------------------------------------------------
def test_sequence_matrix_brute_force():
    rng = C.SplitMix64(7)
    gates = [
        C.Gate("a", (2, 0), C.random_unitary(2, rng)),
        C.Gate("b", (1,), C.random_unitary(1, rng)),
        C.Gate("c", (0, 1, 2), C.random_unitary(3, rng)),
    ]
    # block order [0, 1, 2] coincides with a 3-qubit register, so the brute
    # force product of full unitaries is the expected matrix
    want = np.eye(8, dtype=np.complex128)
    for g in gates:
        want = full_unitary(3, g.qubits, g.matrix) @ want
    np.testing.assert_allclose(oracle.sequence_matrix([0, 1, 2], gates), want, atol=1e-14)
    # a permuted block order is a permutation of rows and columns
    got = oracle.sequence_matrix([2, 0, 1], gates)
    perm = [int(f"{(x >> 1) & 1}{x & 1}{(x >> 2) & 1}", 2) for x in range(8)]
    np.testing.assert_allclose(got, want[np.ix_(perm, perm)], atol=1e-14)


def test_cphase_block_is_diagonal_closed_form():
    """The compress example's first block (0,1,2) holds CPHASE(1) on (0,1),
    (0,2), (1,2): diagonal with phase exp(i * #pairs of set bits)."""
    gates = [C.Gate("CPHASE", p, C.cphase(1.0)) for p in [(0, 1), (0, 2), (1, 2)]]
    m = oracle.sequence_matrix([0, 1, 2], gates)
    for x in range(8):
        b = bin(x).count("1")
        assert m[x, x] == pytest.approx(np.exp(1j * b * (b - 1) / 2))
    assert np.count_nonzero(np.abs(m) > 1e-15) == 8
