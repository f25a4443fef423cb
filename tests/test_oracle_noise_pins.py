"""Pins of the noise oracle (oracle/noise.py) against closed forms, the
state-vector oracle (independent C code) and the paper's depolarizing
figure (Sec. 5): decay of <X> under depolarizing noise during Z rotations."""
import numpy as np
import pytest

import oracle
from oracle import noise as N
from paper_2111_06868_gb300 import circuits as C


def random_rho(n, seed):
    rng = np.random.default_rng(seed)  # input only
    A = rng.standard_normal((1 << n, 1 << n)) + 1j * rng.standard_normal((1 << n, 1 << n))
    rho = A @ A.conj().T
    return rho / np.trace(rho)


def test_embed_matches_state_vector_oracle():
    n = 5
    rng = C.SplitMix64(2)
    psi = oracle.state_init(n, "+-0+1")
    for qs in [(3,), (4, 0), (2, 4, 1), (0, 1, 2, 3, 4)]:
        U = C.random_unitary(len(qs), rng)
        want = oracle.apply_gate(psi.copy(), n, qs, U)
        np.testing.assert_allclose(N.embed(U, n, list(qs)) @ psi, want, atol=1e-14)


def test_partial_trace_replace_on_product_and_bell_states():
    n = 4
    singles = [N.pure_dm(v / np.linalg.norm(v)) for v in
               (np.array([1, 2j]), np.array([3, -1]), np.array([1, 1 + 1j]), np.array([0.5, 2]))]
    rho = singles[0]
    for s in singles[1:]:
        rho = np.kron(rho, s)
    Q = [3, 1]
    want = np.ones((1, 1))
    for q in range(n):
        want = np.kron(want, np.eye(2) / 2 if q in Q else singles[q])
    np.testing.assert_allclose(N.partial_trace_replace(rho, n, Q), want, atol=1e-15)
    bell = np.array([1, 0, 0, 1]) / np.sqrt(2)
    np.testing.assert_allclose(N.partial_trace_replace(N.pure_dm(bell), 2, [1]), np.eye(4) / 4, atol=1e-15)


@pytest.mark.parametrize("qs", [[2], [0, 3], [3, 1]])
def test_depolarizing_closed_form(qs):
    """rho -> (1 - p) rho + p I/d (x) Tr_Q rho (Sec. 2.1 GlobalDepolarizingChannel
    on the qubits Q)."""
    n, p = 4, 0.3
    rho = random_rho(n, len(qs))
    got = N.apply_map(rho, n, qs, N.depolarizing_kraus(p, len(qs)))
    want = (1 - p) * rho + p * N.partial_trace_replace(rho, n, qs)
    np.testing.assert_allclose(got, want, atol=1e-14)


def test_depolarizing_during_z_rotation_figure():
    """|+>, then m steps of RZ(theta) followed by depolarizing p: the Bloch
    vector turns by theta and shrinks by 1 - p each step, so
    <X>_m = (1 - p)^m cos(m theta)."""
    p, theta = 0.05, 0.3
    rho = N.pure_dm(np.array([1, 1]) / np.sqrt(2))
    rz = C.rot("Z", theta)
    for m in range(1, 30):
        rho = N.apply_unitary_dm(rho, 1, [0], rz)
        rho = N.apply_map(rho, 1, [0], N.depolarizing_kraus(p))
        assert abs(N.dm_expectation(rho, [(1.0, ((0, "X"),))]) - (1 - p) ** m * np.cos(m * theta)) <= 1e-14


@pytest.mark.parametrize("e", [0.0, 0.15])
def test_amplitude_damping_closed_form(e):
    g = 0.4
    a, d, b = 0.3, 0.7, 0.2 - 0.35j
    rho = np.array([[a, b], [np.conj(b), d]])
    got = N.apply_map(rho, 1, [0], N.amplitude_damping_kraus(g, e))
    off = np.sqrt((1 - e) * (1 - g)) * b
    want = np.array([[a * (1 - e) + g * d, off], [np.conj(off), d * (1 - g) + e * a]])
    np.testing.assert_allclose(got, want, atol=1e-15)


def test_dephasing_and_general_map():
    p = 0.2
    rho = random_rho(1, 7)
    got = N.apply_map(rho, 1, [0], N.dephasing_kraus(p, "Z"))
    want = rho.copy()
    want[0, 1] *= 1 - 2 * p
    want[1, 0] *= 1 - 2 * p
    np.testing.assert_allclose(got, want, atol=1e-15)
    # the same map as sum_ij s_ij L_i rho R_j^dag with L = R = (I, Z), s diagonal
    I, Z = np.eye(2), np.diag([1.0, -1.0])
    np.testing.assert_allclose(N.apply_map(rho, 1, [0], [I, Z], [I, Z], np.diag([1 - p, p])), want, atol=1e-15)


def test_every_channel_is_trace_preserving():
    sets = [N.depolarizing_kraus(0.3, 1), N.depolarizing_kraus(0.2, 2), N.dephasing_kraus(0.1, "X"),
            N.dephasing_kraus(0.1, "Y"), N.amplitude_damping_kraus(0.3), N.amplitude_damping_kraus(0.3, 0.2)]
    for ks in sets:
        np.testing.assert_allclose(sum(K.conj().T @ K for K in ks), np.eye(ks[0].shape[0]), atol=1e-15)


def test_unitary_map_and_expectation_match_state_vector_oracle():
    n = 4
    rng = C.SplitMix64(3)
    psi = oracle.state_init(n, "+0-1")
    rho = N.pure_dm(psi)
    for qs in [(1, 3), (0,), (2, 0, 3)]:
        U = C.random_unitary(len(qs), rng)
        psi = oracle.apply_gate(psi, n, qs, U)
        rho = N.apply_map(rho, n, list(qs), [U])
    np.testing.assert_allclose(rho, N.pure_dm(psi), atol=1e-14)
    H = [(0.7, ((1, "X"), (2, "Y"))), (-0.4, ((3, "Z"),)), (0.25, ((0, "Y"),))]
    assert abs(N.dm_expectation(rho, H) - oracle.expectation(psi, H)) <= 1e-14


def test_trajectory_branch_choice_and_average():
    """Amplitude damping on |1>: K0 with probability 1 - gamma, K1 with gamma
    (the cumulative threshold decides); the average of <Z> over sampled
    trajectories of a noisy circuit converges to the exact map."""
    g = 0.3
    one = np.array([0, 1], dtype=np.complex128)
    i, out = N.trajectory_step(one, 1, [0], N.amplitude_damping_kraus(g), 0.69)
    assert i == 0 and np.allclose(out, one)
    i, out = N.trajectory_step(one, 1, [0], N.amplitude_damping_kraus(g), 0.71)
    assert i == 1 and np.allclose(out, [1, 0])
    n = 3
    rng = C.SplitMix64(11)
    ops = []
    for layer in range(3):
        for q in range(n):
            ops.append(("U", [q], C.random_unitary(1, rng)))
        ops.append(("U", [layer % n, (layer + 1) % n], C.cz()))
        ops.append(("K", [layer % n], N.amplitude_damping_kraus(0.25)))
        ops.append(("K", [(layer + 2) % n], N.depolarizing_kraus(0.2)))
    rho = N.pure_dm(oracle.state_init(n, "0+1"))
    for kind, qs, m in ops:
        rho = N.apply_unitary_dm(rho, n, qs, m) if kind == "U" else N.apply_map(rho, n, qs, m)
    H = [(1.0, ((0, "Z"),)), (0.5, ((2, "X"),))]
    exact = N.dm_expectation(rho, H)
    u = np.random.default_rng(5)  # input only: the uniforms each step draws
    vals = []
    for _ in range(3000):
        psi = oracle.state_init(n, "0+1")
        for kind, qs, m in ops:
            psi = oracle.apply_gate(psi, n, qs, m) if kind == "U" else N.trajectory_step(psi, n, qs, m, u.random())[1]
        vals.append(oracle.expectation(psi, H))
    vals = np.array(vals)
    assert abs(vals.mean() - exact) <= 5 * vals.std() / np.sqrt(len(vals))


def _random_ops(k, count, rng):
    d = 1 << k
    return [rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d)) for _ in range(count)]


@pytest.mark.parametrize("qs", [[2], [0, 3], [3, 1], [1, 3, 0]])
def test_superop_vectorises_the_general_map(qs):
    """Sec. 5's map sum_ij s_ij L_i rho R_j^dag with random non-Hermitian L, R
    and complex s, through the superoperator S = sum_ij s_ij L_i (x) conj(R_j)
    (row-major vec(A X B) = (A (x) B^T) vec(X), with B = R^dag): a swapped row
    and column order, a missing conjugate or a transposed S each fail here."""
    n = 4
    rng = np.random.default_rng(11 + len(qs))  # input only
    k = len(qs)
    L, R = _random_ops(k, 2, rng), _random_ops(k, 3, rng)
    s = rng.standard_normal((2, 3)) + 1j * rng.standard_normal((2, 3))
    rho = random_rho(n, 5)
    S = sum(s[i, j] * np.kron(L[i], R[j].conj()) for i in range(2) for j in range(3))
    np.testing.assert_allclose(N.apply_superop(rho, n, qs, S), N.apply_map(rho, n, qs, L, R, s), atol=1e-12)


def test_superop_closed_forms():
    """Row/column order of the pair index fixed by maps with a closed form on
    qubit q of a random 3-qubit rho (tensor axes: rows 0..2, columns 3..5)."""
    n, q = 3, 1
    rho = random_rho(n, 8)
    t = rho.reshape((2,) * 6)
    # full depolarization: S = vec(I) vec(I)^T / 2 -> I/2 (x) Tr_q rho
    vI = np.eye(2).reshape(4)
    np.testing.assert_allclose(N.apply_superop(rho, n, [q], np.outer(vI, vI) / 2),
                               N.partial_trace_replace(rho, n, [q]), atol=1e-15)
    # the partial transpose on q: S[(a, b), (c, d)] = [a == d][b == c]
    T = np.zeros((4, 4))
    for a in range(2):
        for b in range(2):
            T[2 * a + b, 2 * b + a] = 1
    want = np.swapaxes(t, q, n + q).reshape(8, 8)
    np.testing.assert_allclose(N.apply_superop(rho, n, [q], T), want, atol=0)
    # S[(0, 1), (0, 0)] = 1: row bit 0 and column bit 1 on q receive the
    # (row 0, column 0) block; everything else becomes 0
    E = np.zeros((4, 4))
    E[1, 0] = 1
    got = N.apply_superop(rho, n, [q], E).reshape((2,) * 6)
    want = np.zeros_like(t)
    idx = [slice(None)] * 6
    src = list(idx)
    src[q], src[n + q] = 0, 0
    dst = list(idx)
    dst[q], dst[n + q] = 0, 1
    want[tuple(dst)] = t[tuple(src)]
    np.testing.assert_allclose(got, want, atol=0)
