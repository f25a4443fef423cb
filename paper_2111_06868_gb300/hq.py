"""Thin ctypes binding of libhq.so (include/hq.h): argument marshalling only.

Every function has the name of the C entry point it calls.  State vectors are
torch tensors (complex64 / complex128, 2^n elements, CUDA, contiguous); the
stream is torch's current stream unless one is given.  Every step of the path
runs in libhq.so's kernels; if the library is missing or a call fails, these
functions raise -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhq.so")

HQ_MAX_K = 6
HQ_MAX_N = 34
HQ_MAX_PAULI = 8
HQ_C64, HQ_C128 = 0, 1
HQ_OP_MATRIX, HQ_OP_ROT = 0, 1
HQ_ENGINE_AUTO, HQ_ENGINE_CUDA_CORE, HQ_ENGINE_TC_F16, HQ_ENGINE_TC_BF16 = 0, 1, 2, 3
ENGINES = {"auto": 0, "cuda_core": 1, "tc_f16": 2, "tc_bf16": 3, "tc_pass": 4, "df": 5, "tc_c128": 6}
PASS_RECORD = 29

STATUS = {
    0: "HQ_OK", -1: "HQ_ERR_NULL", -2: "HQ_ERR_QUBIT_RANGE", -3: "HQ_ERR_DUP_QUBIT", -4: "HQ_ERR_K_TOO_LARGE",
    -5: "HQ_ERR_N_TOO_LARGE", -6: "HQ_ERR_DTYPE", -7: "HQ_ERR_ALLOC", -8: "HQ_ERR_CUDA", -9: "HQ_ERR_TIMEOUT",
    -10: "HQ_ERR_TOKEN", -11: "HQ_ERR_CAPACITY", -12: "HQ_ERR_ARG", -13: "HQ_ERR_ALIGN",
}


class HQError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.name}" + (f" ({detail})" if detail else ""))


class hq_gate(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("qubits", ctypes.c_int * HQ_MAX_K), ("matrix", ctypes.c_void_p)]


class hq_op(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int), ("k", ctypes.c_int), ("qubits", ctypes.c_int * HQ_MAX_K),
        ("matrix", ctypes.c_void_p), ("axis", ctypes.c_int), ("param", ctypes.c_int),
    ]


class hq_pauli_term(ctypes.Structure):
    _fields_ = [
        ("coeff", ctypes.c_double), ("len", ctypes.c_int), ("qubits", ctypes.c_int * HQ_MAX_PAULI),
        ("ops", ctypes.c_char * HQ_MAX_PAULI),
    ]


class hq_noisy_op(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("qubits", ctypes.c_int * HQ_MAX_K), ("nkraus", ctypes.c_int),
                ("matrix", ctypes.c_void_p)]


HQ_DM_MAX_K = 3
HQ_DM_MAP, HQ_DM_SUPER = 0, 1


class hq_dm_op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("k", ctypes.c_int), ("qubits", ctypes.c_int * HQ_DM_MAX_K),
                ("nl", ctypes.c_int), ("nr", ctypes.c_int), ("left", ctypes.c_void_p), ("right", ctypes.c_void_p),
                ("s", ctypes.c_void_p)]


class hq_config(ctypes.Structure):
    _fields_ = [("engine", ctypes.c_int), ("tc_min_k", ctypes.c_int)]


class hq_circuit(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("G", ctypes.c_int), ("gates", ctypes.c_void_p), ("state", ctypes.c_void_p)]


class hq_batch_config(ctypes.Structure):
    _fields_ = [("tile_bits", ctypes.c_int), ("max_high", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("small_first", ctypes.c_int), ("fuse_k", ctypes.c_int)]


_lib = None


def load(path: str | None = None):
    """Load libhq.so (built by ``paper_2111_06868_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build the CUDA library first (paper_2111_06868_gb300.build.build())")
    lib = ctypes.CDLL(p)
    V, I, D, P = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER
    sig = {
        "hq_status_string": ([I], ctypes.c_char_p),
        "hq_last_error": ([], ctypes.c_char_p),
        "hq_version": ([], ctypes.c_char_p),
        "hq_state_init": ([V, I, I, ctypes.c_char_p, V], I),
        "hq_state_upload": ([V, V, I, I, V], I),
        "hq_fuse": ([I, V, I, I, V, P(I), V, ctypes.c_int64, V], I),
        "hq_fuse_dag": ([I, V, I, I, I, ctypes.c_uint64, V, P(I), V, ctypes.c_int64, V], I),
        "hq_fuse_beam": ([I, V, I, I, I, ctypes.c_uint64, V, P(I), V, ctypes.c_int64, V], I),
        "hq_gate_structure": ([I, V, P(I), V], I),
        "hq_pop": ([I, V, I, V, I, I, V], I),
        "hq_reduced_density_matrix": ([V, I, I, V, I, V, V], I),
        "hq_apply_kraus_sampled": ([V, I, I, V, I, I, V, ctypes.c_double, V, V], I),
        "hq_run_trajectory": ([V, I, I, V, I, V, V, V, V], I),
        "hq_simplify": ([I, V, I, I, ctypes.c_double, V], I),
        "hq_test_fail_next_allocs": ([I], I),
        "hq_test_batch_wait_limit_ns": ([ctypes.c_ulonglong], I),
        "hq_dm_superop": ([I, I, V, I, V, V, V], I),
        "hq_dm_init": ([V, I, I, ctypes.c_char_p, V], I),
        "hq_dm_apply": ([V, I, I, V, I, I, V, V], I),
        "hq_dm_expectation": ([V, I, I, V, I, P(D), V], I),
        "hq_dm_purity": ([V, I, I, P(D), V], I),
        "hq_plan_passes": ([I, V, I, I, V, I], I),
        "hq_apply_gate": ([V, I, I, V, I, V, V], I),
        "hq_apply_blocks": ([V, I, I, V, I, V, V], I),
        "hq_simulate": ([V, I, I, ctypes.c_char_p, V, I, V, P(D), V], I),
        "hq_expectation": ([V, I, I, V, I, P(D), V], I),
        "hq_expectation_static": ([V, I, I, V, I, P(D), V], I),
        "hq_adjoint_workspace_bytes": ([I, I, I, I, I, I], ctypes.c_size_t),
        "hq_adjoint_grad": ([I, I, V, I, I, V, I, V, I, ctypes.c_char_p, I, V, ctypes.c_size_t, V, V, V], I),
        "hq_batch_workspace_bytes": ([V, I, V], ctypes.c_size_t),
        "hq_batch_create": ([V, I, V, V, ctypes.c_size_t, V, P(V)], I),
        "hq_batch_run": ([V, V], I),
        "hq_batch_latencies": ([V, V, V, P(D)], I),
        "hq_batch_destroy": ([V], None),
    }
    for name, (args, res) in sig.items():
        if hasattr(lib, name):
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != 0:
        detail = ""
        if st == -8:
            detail = load().hq_last_error().decode()
        raise HQError(st, where, detail)


# ----------------------------------------------------------------------------
# marshalling helpers
# ----------------------------------------------------------------------------
def _dtype_code(t) -> int:
    import torch

    if t.dtype == torch.complex64:
        return HQ_C64
    if t.dtype == torch.complex128:
        return HQ_C128
    raise TypeError(f"state must be complex64 or complex128, got {t.dtype}")


def _state_args(state, nstates: int = 1):
    if not state.is_cuda or not state.is_contiguous():
        raise ValueError("state must be a contiguous CUDA tensor")
    numel = state.numel() // nstates
    n = numel.bit_length() - 1
    if numel != 1 << n:
        raise ValueError("state length must be a power of two")
    return ctypes.c_void_p(state.data_ptr()), n, _dtype_code(state)


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _gate_struct(qubits: Sequence[int], matrix: np.ndarray, keep: list) -> hq_gate:
    m = np.ascontiguousarray(matrix, np.complex128)
    keep.append(m)
    g = hq_gate()
    g.k = len(qubits)
    for j, q in enumerate(qubits):
        g.qubits[j] = int(q)
    g.matrix = m.ctypes.data
    return g


def _gates_array(gates: Iterable, keep: list):
    gl = list(gates)
    arr = (hq_gate * max(1, len(gl)))()
    for i, g in enumerate(gl):
        qs, m = (g.qubits, g.matrix) if hasattr(g, "qubits") else g
        arr[i] = _gate_struct(qs, m, keep)
    return arr, len(gl)


def _terms_array(H) -> tuple:
    arr = (hq_pauli_term * max(1, len(H)))()
    for t, (c, term) in enumerate(H):
        arr[t].coeff = float(c)
        arr[t].len = len(term)
        for j, (q, _) in enumerate(term):
            arr[t].qubits[j] = int(q)
        arr[t].ops = "".join(p for _, p in term).encode()
    return arr, len(H)


# ----------------------------------------------------------------------------
# entry points
# ----------------------------------------------------------------------------
def hq_status_string(st: int) -> str:
    return load().hq_status_string(st).decode()


def hq_version() -> str:
    return load().hq_version().decode()


def hq_state_init(state, tokens: str | None = None, stream=None):
    ptr, n, dt = _state_args(state)
    tok = None
    if tokens is not None:
        tok = (tokens * n if len(tokens) == 1 else tokens).encode()
        if len(tok) != n:
            raise ValueError("need one token per qubit")
    _check(load().hq_state_init(ptr, n, dt, tok, _stream(stream)), "hq_state_init")
    return state


def hq_state_upload(state, host, stream=None):
    """state (CUDA tensor) <- host (CPU tensor of the same dtype and size;
    pinned memory is read by the GPU directly), asynchronously on the stream."""
    ptr, n, dt = _state_args(state)
    if host.is_cuda or not host.is_contiguous() or host.dtype != state.dtype or host.numel() != state.numel():
        raise ValueError("host must be a contiguous CPU tensor of the state's dtype and size")
    _check(load().hq_state_upload(ptr, ctypes.c_void_p(host.data_ptr()), n, dt, _stream(stream)), "hq_state_upload")
    return state


def hq_apply_gate(state, qubits: Sequence[int], matrix, stream=None):
    ptr, n, dt = _state_args(state)
    q = (ctypes.c_int * max(1, len(qubits)))(*[int(x) for x in qubits])
    m = np.ascontiguousarray(matrix, np.complex128)
    _check(load().hq_apply_gate(ptr, n, dt, q, len(qubits), m.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
           "hq_apply_gate")
    return state


def hq_plan_passes(n: int, blocks: Iterable, max_blocks: int = 2):
    """The tile-pass plan (list of dicts: slots, gates, dest) that the
    "tc_pass" engine runs for these blocks; host only."""
    keep: list = []
    arr, G = _gates_array(blocks, keep)
    lib = load()
    cap = 2 * G + 16
    while True:
        rec = np.zeros(cap * PASS_RECORD, np.int32)
        cnt = lib.hq_plan_passes(n, arr, G, max_blocks, rec.ctypes.data_as(ctypes.c_void_p), cap)
        if cnt < 0:
            raise HQError(cnt, "hq_plan_passes", "")
        if cnt <= cap:
            break
        cap = cnt
    out = []
    for i in range(cnt):
        r = rec[i * PASS_RECORD:(i + 1) * PASS_RECORD]
        out.append({"slots": [int(x) for x in r[:13]], "gates": [int(x) for x in r[14:14 + int(r[13])]],
                    "dest": [int(x) for x in r[16:29]]})
    return out


STRUCT_DIAGONAL, STRUCT_MONOMIAL, STRUCT_CONTROLLED = 1, 2, 4
POP_DIRECTIONS = {"right": 0, "left": 1}


def hq_pop(n: int, gates, pinned, direction: str = "right") -> list:
    """The gates (as given) inside the light cone of the pinned qubits."""
    gates = list(gates)
    keep_alive: list = []
    arr, G = _gates_array(gates, keep_alive)
    keep = np.zeros(max(1, G), np.int32)
    pq = np.ascontiguousarray(list(pinned), np.int32)
    r = load().hq_pop(n, arr, G, pq.ctypes.data_as(ctypes.c_void_p), len(pq), POP_DIRECTIONS[direction],
                      keep.ctypes.data_as(ctypes.c_void_p))
    if r < 0:
        _check(r, "hq_pop")
    return [g for g, k in zip(gates, keep[:G]) if k]


def hq_simplify(n: int, gates, use_matrix_commutation: bool = True, atol: float = 1e-12) -> list:
    """The gates (as given) that remain after dropping identities and
    cancelling pairs."""
    gates = list(gates)
    keep_alive: list = []
    arr, G = _gates_array(gates, keep_alive)
    keep = np.zeros(max(1, G), np.int32)
    r = load().hq_simplify(n, arr, G, int(bool(use_matrix_commutation)), float(atol),
                           keep.ctypes.data_as(ctypes.c_void_p))
    if r < 0:
        _check(r, "hq_simplify")
    return [g for g, k in zip(gates, keep[:G]) if k]


def hq_gate_structure(matrix):
    """(structure bits, control mask, matrix on the targets where every control
    is 1) of a 2^k x 2^k matrix, as hq_apply_gate classifies it."""
    m = np.ascontiguousarray(matrix, np.complex128)
    k = int(m.shape[0]).bit_length() - 1
    if m.shape != (1 << k, 1 << k):
        raise ValueError("matrix must be 2^k x 2^k")
    u = np.zeros(2 * 4 ** k, np.float64)
    cm = ctypes.c_int(0)
    s = load().hq_gate_structure(k, m.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cm),
                                 u.ctypes.data_as(ctypes.c_void_p))
    if s < 0:
        _check(s, "hq_gate_structure")
    kt = k - bin(cm.value).count("1")
    d = 1 << kt
    return s, cm.value, u[: 2 * d * d].view(np.complex128).reshape(d, d).copy()


def hq_fuse(n: int, gates: Iterable, k_max: int, with_members: bool = False, method: str = "greedy",
            restarts: int = 64, seed: int = 0, width: int = 128):
    """Returns blocks as a list of (qubits tuple, complex128 matrix).
    method "greedy": hq_fuse; "dag": hq_fuse_dag with `restarts` and `seed`;
    "beam": hq_fuse_beam with `width` and `seed`."""
    keep: list = []
    arr, G = _gates_array(gates, keep)
    cap = max(1, G)
    blocks = (hq_gate * cap)()
    B = ctypes.c_int(cap)
    pool = np.zeros(2 * max(1, G) * (4 ** k_max), np.float64)
    members = np.zeros(max(1, G), np.int32)
    tail = (blocks, ctypes.byref(B), pool.ctypes.data_as(ctypes.c_void_p), pool.size,
            members.ctypes.data_as(ctypes.c_void_p))
    if method == "greedy":
        _check(load().hq_fuse(n, arr, G, k_max, *tail), "hq_fuse")
    elif method == "dag":
        _check(load().hq_fuse_dag(n, arr, G, k_max, restarts, seed, *tail), "hq_fuse_dag")
    elif method == "beam":
        _check(load().hq_fuse_beam(n, arr, G, k_max, width, seed, *tail), "hq_fuse_beam")
    else:
        raise ValueError(f"unknown fusion method {method!r}")
    out = []
    base = pool.ctypes.data
    for i in range(B.value):
        b = blocks[i]
        qs = tuple(b.qubits[j] for j in range(b.k))
        off = (b.matrix - base) // 8
        d = 1 << b.k
        m = pool[off: off + 2 * d * d].view(np.complex128).reshape(d, d).copy()
        out.append((qs, m))
    if with_members:
        return out, members[:G].copy()
    return out


def hq_apply_blocks(state, blocks: Iterable, engine: str | int = "auto", tc_min_k: int = 5, stream=None):
    ptr, n, dt = _state_args(state)
    keep: list = []
    arr, G = _gates_array(blocks, keep)
    cfg = hq_config(ENGINES[engine] if isinstance(engine, str) else int(engine), tc_min_k)
    _check(load().hq_apply_blocks(ptr, n, dt, arr, G, ctypes.byref(cfg), _stream(stream)), "hq_apply_blocks")
    return state


def hq_simulate(state, blocks: Iterable, tokens: str | None = None, engine: str | int = "auto", tc_min_k: int = 5,
                norm: bool = True, stream=None):
    """state <- blocks applied to the product state of `tokens` (None: |0..0>).
    Returns the FP64 squared norm of the result when `norm` (the call then
    synchronises), else None."""
    ptr, n, dt = _state_args(state)
    tok = None
    if tokens is not None:
        tok = (tokens * n if len(tokens) == 1 else tokens).encode()
        if len(tok) != n:
            raise ValueError("need one token per qubit")
    keep: list = []
    arr, G = _gates_array(blocks, keep)
    cfg = hq_config(ENGINES[engine] if isinstance(engine, str) else int(engine), tc_min_k)
    out = ctypes.c_double(0.0)
    _check(load().hq_simulate(ptr, n, dt, tok, arr, G, ctypes.byref(cfg), ctypes.byref(out) if norm else None,
                              _stream(stream)), "hq_simulate")
    return out.value if norm else None


def hq_reduced_density_matrix(state, qubits: Sequence[int], stream=None) -> np.ndarray:
    """Reduced density matrix of 1 or 2 qubits (qubits[0] = MSB of the index)."""
    ptr, n, dt = _state_args(state)
    k = len(qubits)
    q = (ctypes.c_int * max(1, k))(*[int(x) for x in qubits])
    out = np.zeros(2 * 4 ** max(k, 1), np.float64)
    _check(load().hq_reduced_density_matrix(ptr, n, dt, q, k, out.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
           "hq_reduced_density_matrix")
    return out.view(np.complex128).reshape(1 << k, 1 << k)


def _kraus_block(kraus) -> np.ndarray:
    return np.ascontiguousarray(np.stack([np.asarray(K, np.complex128) for K in kraus]), np.complex128)


def hq_apply_kraus_sampled(state, qubits: Sequence[int], kraus, u: float, stream=None) -> int:
    """Sample one Kraus operator of the channel with the uniform u and apply
    it (renormalised); returns its index."""
    ptr, n, dt = _state_args(state)
    k = len(qubits)
    q = (ctypes.c_int * max(1, k))(*[int(x) for x in qubits])
    ks = _kraus_block(kraus)
    chosen = ctypes.c_int(-1)
    _check(load().hq_apply_kraus_sampled(ptr, n, dt, q, k, len(ks), ks.ctypes.data_as(ctypes.c_void_p), float(u),
                                         ctypes.byref(chosen), _stream(stream)), "hq_apply_kraus_sampled")
    return chosen.value


def hq_run_trajectory(state, ops, u, engine: str | int = "auto", tc_min_k: int = 4, stream=None) -> np.ndarray:
    """One trajectory of a noisy circuit.  ops: ("gate", qubits, matrix) or
    ("kraus", qubits, [K_0, ...]); u: one uniform per channel.  Returns the
    sampled Kraus index of every channel."""
    ptr, n, dt = _state_args(state)
    keep: list = []
    arr = (hq_noisy_op * max(1, len(ops)))()
    for i, (kind, qubits, m) in enumerate(ops):
        arr[i].k = len(qubits)
        for j, q in enumerate(qubits):
            arr[i].qubits[j] = int(q)
        if kind == "gate":
            mm = np.ascontiguousarray(m, np.complex128)
            arr[i].nkraus = 0
        elif kind == "kraus":
            mm = _kraus_block(m)
            arr[i].nkraus = len(mm)
        else:
            raise ValueError(f"unknown op kind {kind!r}")
        keep.append(mm)
        arr[i].matrix = mm.ctypes.data
    uu = np.ascontiguousarray(u, np.float64)
    nch = sum(1 for kind, _, _ in ops if kind == "kraus")
    if uu.size < nch:
        raise ValueError("one uniform per channel is needed")
    chosen = np.full(max(1, nch), -1, np.int32)
    cfg = hq_config(ENGINES[engine] if isinstance(engine, str) else int(engine), tc_min_k)
    _check(load().hq_run_trajectory(ptr, n, dt, arr, len(ops), uu.ctypes.data_as(ctypes.c_void_p),
                                    chosen.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cfg), _stream(stream)),
           "hq_run_trajectory")
    return chosen[:nch]


def hq_expectation(state, H, stream=None) -> float:
    ptr, n, dt = _state_args(state)
    arr, T = _terms_array(H)
    out = ctypes.c_double(0.0)
    _check(load().hq_expectation(ptr, n, dt, arr, T, ctypes.byref(out), _stream(stream)), "hq_expectation")
    return out.value


def hq_expectation_static(state, H, stream=None) -> float:
    """hq_expectation without any device allocation (shared static scratch;
    see include/hq.h for its limits and the rule on overlapping calls)."""
    ptr, n, dt = _state_args(state)
    arr, T = _terms_array(H)
    out = ctypes.c_double(0.0)
    st = load().hq_expectation_static(ptr, n, dt, arr, T, ctypes.byref(out), _stream(stream))
    if st == -11:
        raise HQError(st, "hq_expectation_static", load().hq_last_error().decode())
    _check(st, "hq_expectation_static")
    return out.value


def _ops_array(circuit, keep: list):
    arr = (hq_op * max(1, len(circuit.gates)))()
    for i, g in enumerate(circuit.gates):
        op = arr[i]
        op.k = g.k
        for j, q in enumerate(g.qubits):
            op.qubits[j] = int(q)
        if g.matrix is not None:
            m = np.ascontiguousarray(g.matrix, np.complex128)
            keep.append(m)
            op.kind = HQ_OP_MATRIX
            op.matrix = m.ctypes.data
        else:
            op.kind = HQ_OP_ROT
            op.axis = ord(g.axis)
            op.param = int(g.param)
    return arr, len(circuit.gates)


def hq_adjoint_workspace_bytes(n: int, dtype_code: int, G: int, P: int, batch: int, checkpoints: int = 0) -> int:
    return int(load().hq_adjoint_workspace_bytes(n, dtype_code, G, P, batch, checkpoints))


def hq_adjoint_grad(circuit, H, theta, dtype="complex64", tokens: str | None = None, checkpoints: int = 0,
                    workspace=None, stream=None):
    """Energies (batch,) and gradients (batch, P) for theta of shape (batch, P)."""
    import torch

    th = np.ascontiguousarray(np.atleast_2d(theta), np.float64)
    batch, P = th.shape
    if P != circuit.n_params:
        raise ValueError("theta must have circuit.n_params columns")
    dt = HQ_C64 if str(dtype).endswith("64") and "128" not in str(dtype) else HQ_C128
    need = hq_adjoint_workspace_bytes(circuit.n, dt, len(circuit.gates), P, batch, checkpoints)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
    keep: list = []
    ops, G = _ops_array(circuit, keep)
    terms, T = _terms_array(H)
    tok = None
    if tokens is not None:
        tok = (tokens * circuit.n if len(tokens) == 1 else tokens).encode()
    e = np.zeros(batch, np.float64)
    g = np.zeros((batch, max(P, 1)), np.float64)
    _check(load().hq_adjoint_grad(circuit.n, dt, ops, G, P, th.ctypes.data_as(ctypes.c_void_p), batch, terms, T, tok,
                                  checkpoints, ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                  e.ctypes.data_as(ctypes.c_void_p), g.ctypes.data_as(ctypes.c_void_p),
                                  _stream(stream)), "hq_adjoint_grad")
    return e, g[:, :P]


# ----------------------------------------------------------------------------
# batched persistent runs
# ----------------------------------------------------------------------------
def _batch_structs(circuits, states):
    keep: list = []
    arr = (hq_circuit * len(circuits))()
    for i, c in enumerate(circuits):
        garr, G = _gates_array(c.gates, keep)
        keep.append(garr)
        arr[i].n = c.n
        arr[i].G = G
        arr[i].gates = ctypes.cast(garr, ctypes.c_void_p)
        arr[i].state = states[i].data_ptr() if states is not None else (1 << 20) * (i + 1)
    return arr, keep


def hq_batch_workspace_bytes(circuits, tile_bits: int = 0, max_high: int = 0, ctas_per_sm: int = 0,
                             small_first: int = 0, fuse_k: int = 0) -> int:
    arr, keep = _batch_structs(circuits, None)
    cfg = hq_batch_config(tile_bits, max_high, ctas_per_sm, small_first, fuse_k)
    return int(load().hq_batch_workspace_bytes(arr, len(circuits), ctypes.byref(cfg)))


class Batch:
    """hq_batch_create / run / latencies / destroy over torch-owned buffers.
    ``states`` (one complex64 tensor of 2^n per circuit) is allocated if not
    given.  ``fuse_k``: width of the in-pass fused blocks (1..3; 0 = 2)."""

    def __init__(self, circuits, states=None, tile_bits: int = 0, max_high: int = 0, ctas_per_sm: int = 0,
                 small_first: int = 0, fuse_k: int = 0, stream=None):
        import torch

        self.circuits = list(circuits)
        if states is None:
            states = [torch.empty(1 << c.n, dtype=torch.complex64, device="cuda") for c in self.circuits]
        self.states = states
        self.cfg = hq_batch_config(tile_bits, max_high, ctas_per_sm, small_first, fuse_k)
        arr, keep = _batch_structs(self.circuits, states)
        need = load().hq_batch_workspace_bytes(arr, len(self.circuits), ctypes.byref(self.cfg))
        if need == 0:
            # the planner refused the input: let hq_batch_create report why
            need = 256
        self.workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        self._h = None
        _check(load().hq_batch_create(arr, len(self.circuits), ctypes.byref(self.cfg),
                                      ctypes.c_void_p(self.workspace.data_ptr()), need, _stream(stream),
                                      ctypes.byref(h)), "hq_batch_create")
        self._h = h
        self.gates = sum(len(c.gates) for c in self.circuits)

    def run(self, stream=None):
        _check(load().hq_batch_run(self._h, _stream(stream)), "hq_batch_run")

    def latencies(self, stream=None):
        lat = np.zeros(len(self.circuits), np.float32)
        mk = ctypes.c_double()
        _check(load().hq_batch_latencies(self._h, _stream(stream), lat.ctypes.data_as(ctypes.c_void_p),
                                         ctypes.byref(mk)), "hq_batch_latencies")
        return lat, mk.value

    def close(self):
        if self._h is not None:
            load().hq_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# density matrices: rho (2^n x 2^n) as the 2n-qubit vector vec(rho), row-major
# ----------------------------------------------------------------------------
def _dm_args(rho):
    ptr, n2, dt = _state_args(rho.reshape(-1))
    if n2 % 2:
        raise ValueError("a density matrix has 4^n entries")
    return ptr, n2 // 2, dt


def _ops_block(ops) -> np.ndarray:
    return np.ascontiguousarray(np.stack([np.asarray(m, np.complex128) for m in ops]), np.complex128)


def hq_dm_superop(left, right=None, s=None) -> np.ndarray:
    """S = sum_ij s_ij L_i (x) conj(R_j) (4^k x 4^k) of the map
    rho -> sum_ij s_ij L_i rho R_j^dag; right None: R = L; s None: identity."""
    L = _ops_block(left)
    k = int(L.shape[1]).bit_length() - 1
    R = None if right is None else _ops_block(right)
    sc = None if s is None else np.ascontiguousarray(s, np.complex128)
    out = np.zeros((4 ** k, 4 ** k), np.complex128)
    _check(load().hq_dm_superop(k, len(L), L.ctypes.data_as(ctypes.c_void_p), 0 if R is None else len(R),
                                None if R is None else R.ctypes.data_as(ctypes.c_void_p),
                                None if sc is None else sc.ctypes.data_as(ctypes.c_void_p),
                                out.ctypes.data_as(ctypes.c_void_p)), "hq_dm_superop")
    return out


def hq_dm_init(rho, tokens: str | None = None, stream=None):
    ptr, n, dt = _dm_args(rho)
    tok = None
    if tokens is not None:
        tok = (tokens * n if len(tokens) == 1 else tokens).encode()
        if len(tok) != n:
            raise ValueError("need one token per qubit")
    _check(load().hq_dm_init(ptr, n, dt, tok, _stream(stream)), "hq_dm_init")
    return rho


def hq_dm_apply(rho, ops, k_max: int = 6, engine: str | int = "auto", tc_min_k: int = 4, stream=None):
    """rho <- the operations in order.  ops: ("gate", qubits, U),
    ("kraus", qubits, [K_0, ...]), ("map", qubits, (L list, R list or None,
    s or None)) or ("super", qubits, S)."""
    ptr, n, dt = _dm_args(rho)
    ops = list(ops)
    arr = (hq_dm_op * max(1, len(ops)))()
    keep: list = []
    for i, (kind, qs, m) in enumerate(ops):
        o = arr[i]
        o.k = len(qs)
        for j, q in enumerate(qs):
            o.qubits[j] = int(q)
        if kind == "super":
            o.kind = HQ_DM_SUPER
            S = np.ascontiguousarray(m, np.complex128)
            keep.append(S)
            o.left = S.ctypes.data
            continue
        o.kind = HQ_DM_MAP
        if kind == "gate":
            L, R, sc = [m], None, None
        elif kind == "kraus":
            L, R, sc = m, None, None
        elif kind == "map":
            L, R, sc = m
        else:
            raise ValueError(f"unknown operation {kind!r}")
        Lb = _ops_block(L)
        keep.append(Lb)
        o.nl, o.left = len(Lb), Lb.ctypes.data
        if R is not None:
            Rb = _ops_block(R)
            keep.append(Rb)
            o.nr, o.right = len(Rb), Rb.ctypes.data
        if sc is not None:
            sb = np.ascontiguousarray(sc, np.complex128)
            keep.append(sb)
            o.s = sb.ctypes.data
    cfg = hq_config(ENGINES[engine] if isinstance(engine, str) else int(engine), tc_min_k)
    _check(load().hq_dm_apply(ptr, n, dt, arr, len(ops), int(k_max), ctypes.byref(cfg), _stream(stream)),
           "hq_dm_apply")
    return rho


def hq_dm_expectation(rho, H, stream=None) -> float:
    """Tr(rho H) for H = [(coeff, ((qubit, 'X'|'Y'|'Z'), ...)), ...]."""
    ptr, n, dt = _dm_args(rho)
    arr, T = _terms_array(H)
    out = ctypes.c_double(0.0)
    _check(load().hq_dm_expectation(ptr, n, dt, arr, T, ctypes.byref(out), _stream(stream)), "hq_dm_expectation")
    return out.value


def hq_dm_purity(rho, stream=None) -> float:
    ptr, n, dt = _dm_args(rho)
    out = ctypes.c_double(0.0)
    _check(load().hq_dm_purity(ptr, n, dt, ctypes.byref(out), _stream(stream)), "hq_dm_purity")
    return out.value


def hq_test_fail_next_allocs(count: int) -> None:
    """Make the library's next `count` device scratch allocations fail
    (HQ_ERR_ALLOC), for tests of the error paths; 0 turns it off."""
    _check(load().hq_test_fail_next_allocs(int(count)), "hq_test_fail_next_allocs")


def hq_test_batch_wait_limit_ns(ns: int) -> None:
    """Let the batch runner's scheduler give up after `ns` nanoseconds without
    work (HQ_ERR_TIMEOUT at the next hq_batch_latencies), for tests of the
    bounded-wait path; 0 restores the 2 s default."""
    _check(load().hq_test_batch_wait_limit_ns(int(ns)), "hq_test_batch_wait_limit_ns")
