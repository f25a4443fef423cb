"""CPU oracle for the state-vector path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, complex128 C implementation (``hq_oracle.c``) of what the GPU
path computes, loaded through ctypes.  Only the tests, the bench's CPU-baseline
leg and the smoke check may import this package; the product never does, and it
shares no code with the CUDA path.

What each function follows (HybridQ, arXiv 2111.06868):
  * ``state_init``        -- Sec. 4.1, product state from '0' '1' '+' '-' tokens.
  * ``apply_gate`` / ``simulate`` -- Sec. 2 (MatrixGate) and Sec. 4.2 (state
    vector evolution): U_G ... U_1 |psi0>, applied gate by gate, unfused.
  * ``sequence_matrix``   -- Sec. 3.1 ``matrix(circuit)``: the matrix of a gate
    sequence on a qubit subset, column by column.
  * ``expectation``       -- <psi|H|psi> for a Pauli sum, factor-by-factor.
  * ``adjoint_grad`` / ``param_shift_grad`` -- dE/dtheta for rotation gates
    (not in the paper; Jones & Gacon adjoint sweep, and the exact
    parameter-shift rule).

Every function is pinned by ``tests/test_oracle_pins.py`` against closed forms,
brute force and the paper's printed examples.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hq_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
# Test hook: a prebuilt library to load instead (the mutation test points this
# at deliberately broken copies to show that the pins catch them).
_OVERRIDE = os.environ.get("HQ_ORACLE_LIB")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (C99 complex, OpenMP for the gate loop)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if _OVERRIDE:
                lib = ctypes.CDLL(_OVERRIDE)
            else:
                build()
                lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i = ctypes.c_int
            lib.or_state_init.argtypes = [i, ctypes.c_char_p, P]
            lib.or_apply_gate.argtypes = [i, P, i, P, P]
            lib.or_apply_circuit.argtypes = [i, P, i, P, P, P, P, P, P, P, P]
            lib.or_expectation.argtypes = [i, P, i, P, P, P, P]
            lib.or_expectation.restype = ctypes.c_double
            lib.or_norm2.argtypes = [i, P]
            lib.or_norm2.restype = ctypes.c_double
            lib.or_energy.argtypes = [i, ctypes.c_char_p, i, P, P, P, P, P, P, P, P, i, P, P, P, P]
            lib.or_energy.restype = ctypes.c_double
            lib.or_adjoint_grad.argtypes = [i, ctypes.c_char_p, i, P, P, P, P, P, P, P, P, i, i, P, P, P, P, P]
            lib.or_adjoint_grad.restype = ctypes.c_double
            lib.or_param_shift_grad.argtypes = [i, ctypes.c_char_p, i, P, P, P, P, P, P, P, P, i, i, P, P, P, P, P]
            lib.or_sequence_matrix.argtypes = [i, P, i, P, P, P, P, P]
            lib.or_set_threads.argtypes = [i]
            lib.or_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _tok(n: int, tokens):
    if tokens is None:
        return None
    if len(tokens) == 1:
        tokens = tokens * n
    if len(tokens) != n:
        raise ValueError("need one token per qubit")
    return tokens.encode()


def set_threads(t: int) -> None:
    _load().or_set_threads(int(t))


def max_threads() -> int:
    return int(_load().or_max_threads())


def state_init(n: int, tokens=None) -> np.ndarray:
    psi = np.empty(1 << n, np.complex128)
    _load().or_state_init(n, _tok(n, tokens), _ptr(psi))
    return psi


def apply_gate(psi: np.ndarray, n: int, qubits, matrix) -> np.ndarray:
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == 1 << n
    q = np.ascontiguousarray(qubits, np.int32)
    m = np.ascontiguousarray(matrix, np.complex128)
    assert m.shape == (1 << len(q), 1 << len(q))
    _load().or_apply_gate(n, _ptr(psi), len(q), _ptr(q), _ptr(m))
    return psi


class _Packed:
    def __init__(self, circuit):
        p = circuit.packed()
        self.G = len(circuit.gates)
        self.k = p["k"]
        self.qubits = np.ascontiguousarray(p["qubits"].ravel())
        self.kind = p["kind"]
        self.axis = p["axis"]
        self.param = p["param"]
        self.mats = np.ascontiguousarray(p["matrices"])
        if self.mats.size == 0:
            self.mats = np.zeros(1, np.complex128)
        self.off = p["offsets"]

    def args(self):
        return (self.G, _ptr(self.k), _ptr(self.qubits), _ptr(self.kind), _ptr(self.axis),
                _ptr(self.param), _ptr(self.mats), _ptr(self.off))


class _Ham:
    def __init__(self, H):
        T = len(H)
        self.T = T
        self.coeff = np.zeros(max(T, 1), np.float64)
        self.len = np.zeros(max(T, 1), np.int32)
        self.q = np.zeros((max(T, 1), 8), np.int32)
        self.op = np.zeros((max(T, 1), 8), np.uint8)
        for t, (c, term) in enumerate(H):
            self.coeff[t] = c
            self.len[t] = len(term)
            for j, (q, p) in enumerate(term):
                self.q[t, j] = q
                self.op[t, j] = ord(p)

    def args(self):
        return (self.T, _ptr(self.coeff), _ptr(self.len), _ptr(self.q), _ptr(self.op))


def _theta(circuit, theta):
    if theta is None:
        theta = np.zeros(max(circuit.n_params, 1))
    return np.ascontiguousarray(theta, np.float64)


def apply_circuit(psi: np.ndarray, circuit, theta=None) -> np.ndarray:
    assert psi.dtype == np.complex128 and psi.size == 1 << circuit.n
    pk = _Packed(circuit)
    th = _theta(circuit, theta)
    _load().or_apply_circuit(circuit.n, _ptr(psi), *pk.args(), _ptr(th))
    return psi


def simulate(circuit, tokens=None, theta=None) -> np.ndarray:
    psi = state_init(circuit.n, tokens)
    return apply_circuit(psi, circuit, theta)


def norm2(psi: np.ndarray) -> float:
    n = int(psi.size).bit_length() - 1
    return float(_load().or_norm2(n, _ptr(np.ascontiguousarray(psi, np.complex128))))


def expectation(psi: np.ndarray, H) -> float:
    n = int(psi.size).bit_length() - 1
    h = _Ham(H)
    return float(_load().or_expectation(n, _ptr(np.ascontiguousarray(psi, np.complex128)), *h.args()))


def energy(circuit, H, theta, tokens=None) -> float:
    pk, h, th = _Packed(circuit), _Ham(H), _theta(circuit, theta)
    return float(_load().or_energy(circuit.n, _tok(circuit.n, tokens), *pk.args(), _ptr(th), *h.args()))


def adjoint_grad(circuit, H, theta, tokens=None):
    pk, h, th = _Packed(circuit), _Ham(H), _theta(circuit, theta)
    g = np.zeros(max(circuit.n_params, 1), np.float64)
    e = _load().or_adjoint_grad(circuit.n, _tok(circuit.n, tokens), *pk.args(), _ptr(th),
                                circuit.n_params, *h.args(), _ptr(g))
    return float(e), g[: circuit.n_params]


def param_shift_grad(circuit, H, theta, tokens=None):
    pk, h, th = _Packed(circuit), _Ham(H), _theta(circuit, theta)
    g = np.zeros(max(circuit.n_params, 1), np.float64)
    _load().or_param_shift_grad(circuit.n, _tok(circuit.n, tokens), *pk.args(), _ptr(th),
                                circuit.n_params, *h.args(), _ptr(g))
    return g[: circuit.n_params]


def sequence_matrix(block_qubits, gates) -> np.ndarray:
    """Matrix (in the order of ``block_qubits``, first = MSB) of the fixed-matrix
    gate sequence ``gates`` (each acting inside ``block_qubits``)."""
    bq = np.ascontiguousarray(block_qubits, np.int32)
    kb = len(bq)
    G = len(gates)
    ks = np.array([len(g.qubits) for g in gates], np.int32)
    qs = np.full((G, 6), -1, np.int32)
    offs = np.zeros(G, np.int64)
    mats, off = [], 0
    for i, g in enumerate(gates):
        qs[i, : len(g.qubits)] = g.qubits
        m = np.ascontiguousarray(g.matrix, np.complex128).ravel()
        mats.append(m)
        offs[i] = off
        off += m.size
    mat = np.concatenate(mats) if mats else np.zeros(1, np.complex128)
    qs = np.ascontiguousarray(qs.ravel())
    out = np.empty((1 << kb, 1 << kb), np.complex128)
    _load().or_sequence_matrix(kb, _ptr(bq), G, _ptr(ks), _ptr(qs), _ptr(mat), _ptr(offs), _ptr(out))
    return out
