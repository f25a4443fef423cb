"""Noise oracle -- TEST INFRASTRUCTURE ONLY.

Plain numpy complex128 implementations, written from the definitions in
HybridQ (arXiv 2111.06868), of what the noisy-simulation paths compute.  Only
the tests and the bench's CPU legs import this module; it shares no code with
the CUDA path or its Python binding.

  * Channels of Sec. 2.1 ("Noisy gates") as Kraus sets:
      - ``depolarizing_kraus(p, k)``: rho -> (1 - p) rho + p I/d (d = 2^k, on
        the k qubits it acts on), written as the Pauli twirl;
      - ``dephasing_kraus(p, sigma)``: rho -> (1 - p) rho + p sigma rho sigma;
      - ``amplitude_damping_kraus(gamma, excitation)``: |0><0| +
        sqrt(1 - gamma)|1><1| and sqrt(gamma)|0><1|, and with a non-zero
        excitation rate e for |0> -> |1> the two-rate form (reading below).
  * ``apply_map(rho, n, qubits, L, R, s)``: the general map of Sec. 5,
    Lambda[X] = sum_ij s_ij L_i X R_j^dag, every operator embedded on
    ``qubits`` of an n-qubit register as a full 2^n x 2^n matrix.
  * ``apply_superop(rho, n, qubits, S)``: the MatrixSuperGate of Sec. 2 --
    rho vectorised and multiplied by a 4^k x 4^k matrix S on the entries
    rho[(a, y), (b, z)] with a, b the local row and column indices of the k
    qubits (pair index a 2^k + b, qubits[0] the most significant bit of a and
    of b) and y, z those of the other qubits, which S leaves alone.
  * ``dm_expectation(rho, H)``: Tr(rho H) for a Pauli sum, H built as an
    explicit Kronecker product.
  * ``trajectory_step(psi, n, qubits, kraus, u)``: one step of the pure-state
    sampling of Kraus operators of Sec. 5: p_i = ||K_i psi||^2, the first i
    whose cumulative probability exceeds u, psi -> K_i psi / sqrt(p_i).

Reading (the paper names the excitation rate but gives no Kraus form): with
decay rate gamma and excitation rate e, K0 = sqrt(1 - e)|0><0| +
sqrt(1 - gamma)|1><1|, K1 = sqrt(gamma)|0><1|, K2 = sqrt(e)|1><0|, which is
trace preserving and reduces to the paper's two operators at e = 0.

Pinned by ``tests/test_oracle_noise_pins.py``: the depolarizing closed form
(through a partial trace), the decay of <X> under depolarizing noise during Z
rotations (the paper's depolarizing figure), amplitude-damping closed forms,
trace preservation, unitary maps against the state-vector oracle, the
trajectory average against the exact map, and the superoperator against the
map it vectorises (row-major vec(A X B) = (A (x) B^T) vec(X)) and against
closed forms that fix its row/column order.
"""
from __future__ import annotations

import itertools

import numpy as np

_PAULI = {
    "I": np.eye(2, dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def _kron_all(ops):
    out = np.ones((1, 1), dtype=np.complex128)
    for o in ops:
        out = np.kron(out, o)
    return out


def embed(op, n, qubits):
    """op (on ``qubits``, first = most significant) as a 2^n x 2^n matrix on
    an n-qubit register whose qubit 0 is the most significant bit."""
    k = len(qubits)
    full = np.kron(op, np.eye(1 << (n - k), dtype=np.complex128))  # op on qubits 0..k-1
    rest = [q for q in range(n) if q not in qubits]
    order = list(qubits) + rest  # register axis order of `full`'s axes
    t = full.reshape((2,) * (2 * n))
    inv = np.argsort(order)
    t = t.transpose(list(inv) + [n + i for i in inv])
    return t.reshape(1 << n, 1 << n)


# ----------------------------------------------------------------------------
# channels (Sec. 2.1)
# ----------------------------------------------------------------------------
def depolarizing_kraus(p: float, k: int = 1):
    """rho -> (1 - p) rho + p I/d on k qubits: the Pauli twirl
    (1/4^k) sum_P P rho P equals I/d (x) Tr_Q rho, so the Kraus operators are
    sqrt(1 - p + p/4^k) I and sqrt(p/4^k) P for the 4^k - 1 other Paulis."""
    ops = []
    for labels in itertools.product("IXYZ", repeat=k):
        P = _kron_all(_PAULI[c] for c in labels)
        w = (1 - p + p / 4 ** k) if set(labels) == {"I"} else p / 4 ** k
        ops.append(np.sqrt(w) * P)
    return ops


def dephasing_kraus(p: float, sigma: str = "Z"):
    return [np.sqrt(1 - p) * _PAULI["I"], np.sqrt(p) * _PAULI[sigma]]


def amplitude_damping_kraus(gamma: float, excitation: float = 0.0):
    K0 = np.array([[np.sqrt(1 - excitation), 0], [0, np.sqrt(1 - gamma)]], dtype=np.complex128)
    K1 = np.array([[0, np.sqrt(gamma)], [0, 0]], dtype=np.complex128)
    ops = [K0, K1]
    if excitation:
        ops.append(np.array([[0, 0], [np.sqrt(excitation), 0]], dtype=np.complex128))
    return ops


# ----------------------------------------------------------------------------
# density matrices (Sec. 5)
# ----------------------------------------------------------------------------
def pure_dm(psi):
    return np.outer(psi, psi.conj())


def apply_map(rho, n, qubits, L, R=None, s=None):
    """Lambda[rho] = sum_ij s_ij L_i rho R_j^dag; R = L and s = I (a Kraus
    map) when omitted."""
    if R is None:
        R = L
    if s is None:
        s = np.eye(len(L))
    Le = [embed(l, n, qubits) for l in L]
    Re = [embed(r, n, qubits) for r in R]
    out = np.zeros_like(rho)
    for i, li in enumerate(Le):
        for j, rj in enumerate(Re):
            if s[i][j] != 0:
                out += s[i][j] * (li @ rho @ rj.conj().T)
    return out


def apply_superop(rho, n, qubits, S):
    """rho' = S acting on vec(rho) (MatrixSuperGate, Sec. 2): for every pair
    (y, z) of indices of the other qubits, the 4^k entries rho[(a, y), (b, z)]
    form a vector indexed by a 2^k + b, and S multiplies it."""
    k = len(qubits)
    rest = [q for q in range(n) if q not in qubits]
    order = list(qubits) + [n + q for q in qubits] + rest + [n + q for q in rest]
    t = rho.reshape((2,) * (2 * n)).transpose(order).reshape(4 ** k, -1)
    t = (np.asarray(S, dtype=np.complex128) @ t).reshape((2,) * (2 * n))
    return t.transpose(np.argsort(order)).reshape(1 << n, 1 << n)


def apply_unitary_dm(rho, n, qubits, U):
    Ue = embed(U, n, qubits)
    return Ue @ rho @ Ue.conj().T


def pauli_matrix(n, term):
    ops = [_PAULI["I"]] * n
    for q, c in term:
        ops[q] = _PAULI[c]
    return _kron_all(ops)


def dm_expectation(rho, H) -> float:
    """Tr(rho H) for H = sum_t c_t P_t (real part; H is Hermitian)."""
    n = int(rho.shape[0]).bit_length() - 1
    return float(sum(c * np.trace(rho @ pauli_matrix(n, term)).real for c, term in H))


def partial_trace_replace(rho, n, qubits):
    """I/d (x) Tr_Q rho: the qubits Q traced out and replaced by the maximally
    mixed state (used to pin the depolarizing channel)."""
    k = len(qubits)
    rest = [q for q in range(n) if q not in qubits]
    t = rho.reshape((2,) * (2 * n))
    order = list(qubits) + rest
    t = t.transpose(order + [n + q for q in order]).reshape(1 << k, 1 << (n - k), 1 << k, 1 << (n - k))
    red = np.einsum("aiaj->ij", t)  # Tr_Q
    full = np.kron(np.eye(1 << k) / (1 << k), red).reshape((2,) * (2 * n))
    inv = np.argsort(order)
    return full.transpose(list(inv) + [n + i for i in inv]).reshape(1 << n, 1 << n)


# ----------------------------------------------------------------------------
# pure-state sampling (Sec. 5)
# ----------------------------------------------------------------------------
def trajectory_step(psi, n, qubits, kraus, u):
    """One sampled Kraus operator: returns (index, new state)."""
    outs = [embed(K, n, qubits) @ psi for K in kraus]
    p = np.array([np.vdot(o, o).real for o in outs])
    i = int(np.searchsorted(np.cumsum(p), u * p.sum(), side="right"))
    i = min(i, len(kraus) - 1)
    return i, outs[i] / np.sqrt(p[i])
