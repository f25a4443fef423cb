"""Host-side checks of libhq.so: it builds, loads without a GPU, exports every
entry point include/hq.h declares, validates arguments, and its host-only
fusion (hq_fuse) reproduces the paper's compress example and is exact."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2111_06868_gb300 import circuits as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hq():
    from paper_2111_06868_gb300 import build
    from paper_2111_06868_gb300 import hq as _hq

    build.build()
    _hq.load()
    return _hq


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hq.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hq_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(hq):
    syms = declared_symbols()
    assert "hq_apply_gate" in syms and "hq_fuse" in syms and "hq_adjoint_grad" in syms
    lib = hq.load()
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_status_strings_and_version(hq):
    assert hq.hq_status_string(0) == "ok"
    for code in hq.STATUS:
        assert hq.hq_status_string(code) != "unknown status"
    assert "sm_103a" in hq.hq_version()


def test_validation_before_any_device_work(hq):
    """Errors that are decided on the host return without touching CUDA."""
    lib = hq.load()
    c_int = hq.ctypes.c_int
    m = np.eye(2, dtype=np.complex128)
    q = (c_int * 1)(0)
    mp = m.ctypes.data_as(hq.ctypes.c_void_p)
    assert lib.hq_apply_gate(None, 4, 0, q, 1, mp, None) == -1            # NULL state
    fake = hq.ctypes.c_void_p(1 << 20)
    assert lib.hq_apply_gate(fake, 0, 0, q, 1, mp, None) == -5            # n too small
    assert lib.hq_apply_gate(fake, 35, 0, q, 1, mp, None) == -5           # n too large
    assert lib.hq_apply_gate(fake, 4, 7, q, 1, mp, None) == -6            # dtype
    assert lib.hq_apply_gate(fake, 4, 0, (c_int * 1)(4), 1, mp, None) == -2  # qubit range
    assert lib.hq_apply_gate(fake, 4, 0, (c_int * 2)(1, 1), 2, mp, None) == -3  # duplicate
    assert lib.hq_apply_gate(fake, 4, 0, (c_int * 7)(*range(7)), 7, mp, None) == -4  # k > 6
    assert lib.hq_apply_gate(fake, 2, 0, (c_int * 3)(0, 1, 2), 3, mp, None) == -4  # k > n
    assert lib.hq_apply_gate(hq.ctypes.c_void_p((1 << 20) + 8), 4, 0, q, 1, mp, None) == -13  # alignment
    assert lib.hq_state_init(fake, 3, 0, b"0x1", None) == -10             # token
    assert lib.hq_apply_gate(fake, 4, 0, q, 1, None, None) == -1          # NULL matrix
    term = hq.hq_pauli_term()
    term.len = 1
    term.qubits[0] = 0
    term.ops = b"Q"
    out = hq.ctypes.c_double()
    assert lib.hq_expectation(fake, 4, 0, hq.ctypes.byref(term), 1, hq.ctypes.byref(out), None) == -12


def paper_compress_circuit():
    return C.Circuit(5, [C.Gate("CPHASE", (q1, q2), C.cphase(1.0)) for q1 in range(5) for q2 in range(q1 + 1, 5)])


def test_fuse_reproduces_compress_example(hq):
    """Sec. 3.1: CPHASE on all pairs of 5 qubits, max_n_qubits=3."""
    want = [tuple(int(x) for x in l.split()) for l in open(os.path.join(ROOT, "tests", "golden", "compress_sec3_1.txt"))
            if l.strip() and not l.startswith("#")]
    circ = paper_compress_circuit()
    blocks = hq.hq_fuse(5, circ.gates, 3)
    assert [q for q, _ in blocks] == want


@pytest.mark.parametrize("method", ["greedy", "dag"])
@pytest.mark.parametrize("kmax", [1, 2, 3, 4, 5, 6])
def test_fused_blocks_equal_their_members(hq, kmax, method):
    """Every block matrix equals the oracle's matrix of its member sequence,
    and the fused circuit leaves the same state as the unfused one."""
    circ = C.random_dense_circuit(8, 40, seed=kmax, kmax=min(kmax, 3))
    blocks, members = hq.hq_fuse(8, circ.gates, kmax, with_members=True, method=method, restarts=8)
    assert all(len(q) <= kmax for q, _ in blocks)
    assert sorted(set(members.tolist())) == list(range(len(blocks)))
    for b, (qs, m) in enumerate(blocks):
        assert list(qs) == sorted(qs)
        mem = [circ.gates[i] for i in range(len(circ.gates)) if members[i] == b]
        np.testing.assert_allclose(m, oracle.sequence_matrix(qs, mem), atol=1e-13)
    psi0 = oracle.state_init(8, "+-01+-01")
    fused = C.Circuit(8, [C.Gate("B", q, m) for q, m in blocks])
    np.testing.assert_allclose(oracle.apply_circuit(psi0.copy(), fused), oracle.apply_circuit(psi0.copy(), circ),
                               atol=1e-12)


def per_qubit_block_order_kept(n, gates, members):
    """Along every qubit, the blocks of its gates never go back: the fused
    circuit is a reordering of the DAG that keeps every qubit's gate order."""
    last = [-1] * n
    for g, b in zip(gates, members):
        for q in g.qubits:
            if b < last[q]:
                return False
            last[q] = b
    return True


@pytest.mark.parametrize("seed", range(4))
def test_fuse_dag_keeps_qubit_order_and_state(hq, seed):
    circ = C.random_circuit(C.grid(3, 4), 12, seed=seed, two_qubit="fsim" if seed % 2 else "cz")
    for kmax in (3, 4, 6):
        blocks, members = hq.hq_fuse(12, circ.gates, kmax, with_members=True, method="dag", restarts=16,
                                     seed=seed)
        assert per_qubit_block_order_kept(12, circ.gates, members)
        assert all(len(q) <= kmax for q, _ in blocks)
        psi0 = oracle.state_init(12, "+-+0-+-1+-+-")
        fused = C.Circuit(12, [C.Gate("B", q, m) for q, m in blocks])
        np.testing.assert_allclose(oracle.apply_circuit(psi0.copy(), fused),
                                   oracle.apply_circuit(psi0.copy(), circ), atol=1e-12)


def test_fuse_dag_is_deterministic_and_not_worse(hq):
    """Fewer blocks than the greedy rule on the grid circuits (n=30: 61 -> 43
    at k_max = 6), and the same blocks for the same seed."""
    for circ, bound in [(C.config_n30(0), 45), (C.config_n33(0), 60)]:
        greedy = hq.hq_fuse(circ.n, circ.gates, 6)
        dag = hq.hq_fuse(circ.n, circ.gates, 6, method="dag")
        assert len(dag) <= bound < len(greedy)
        again = hq.hq_fuse(circ.n, circ.gates, 6, method="dag")
        assert [q for q, _ in again] == [q for q, _ in dag]
        assert all(np.array_equal(a, b) for (_, a), (_, b) in zip(again, dag))
        one = hq.hq_fuse(circ.n, circ.gates, 6, method="dag", restarts=1)
        assert len(dag) <= len(one)


@pytest.mark.parametrize("seed", range(4))
def test_fuse_beam_keeps_qubit_order_and_state(hq, seed):
    circ = C.random_circuit(C.grid(3, 4), 12, seed=seed, two_qubit="fsim" if seed % 2 else "cz")
    for kmax, width in ((3, 8), (4, 32), (6, 128)):
        blocks, members = hq.hq_fuse(12, circ.gates, kmax, with_members=True, method="beam", width=width,
                                     seed=seed)
        assert per_qubit_block_order_kept(12, circ.gates, members)
        assert all(len(q) <= kmax for q, _ in blocks)
        assert sorted(set(members.tolist())) == list(range(len(blocks)))  # every block holds a gate
        psi0 = oracle.state_init(12, "+-+0-+-1+-+-")
        fused = C.Circuit(12, [C.Gate("B", q, m) for q, m in blocks])
        np.testing.assert_allclose(oracle.apply_circuit(psi0.copy(), fused),
                                   oracle.apply_circuit(psi0.copy(), circ), atol=1e-12)


def test_fuse_beam_is_deterministic_and_not_worse(hq):
    """The beam search places fewer blocks than the frontier restarts on the
    grid circuits (n=30: 43 -> 39, n=33: 57 -> 53 at k_max = 6, width 128),
    never more than the frontier rule's first run, and the same blocks for
    the same arguments."""
    for circ, bound in [(C.config_n30(0), 40), (C.config_n33(0), 54)]:
        beam = hq.hq_fuse(circ.n, circ.gates, 6, method="beam", width=128)
        one = hq.hq_fuse(circ.n, circ.gates, 6, method="dag", restarts=1)
        dag = hq.hq_fuse(circ.n, circ.gates, 6, method="dag")
        assert len(beam) <= bound < len(dag) <= len(one)
        again = hq.hq_fuse(circ.n, circ.gates, 6, method="beam", width=128)
        assert [q for q, _ in again] == [q for q, _ in beam]
        assert all(np.array_equal(a, b) for (_, a), (_, b) in zip(again, beam))
    # width 1 is the frontier rule with four proposals per frontier gate
    circ = C.config_n30(0)
    assert len(hq.hq_fuse(30, circ.gates, 6, method="beam", width=1)) <= len(one)


def test_fuse_beam_errors_and_empty(hq):
    circ = C.Circuit(4, [C.Gate("U", (0, 1, 2), np.eye(8, dtype=np.complex128))])
    for w in (0, 4097):
        with pytest.raises(hq.HQError, match="ARG"):
            hq.hq_fuse(4, circ.gates, 3, method="beam", width=w)
    with pytest.raises(hq.HQError, match="K_TOO_LARGE"):
        hq.hq_fuse(4, circ.gates, 2, method="beam")
    assert hq.hq_fuse(3, [], 4, method="beam") == []


def test_fuse_grid_circuit_reduces_passes(hq):
    circ = C.config_n30(0)
    for kmax, bound in [(2, 845), (4, 300), (6, 200)]:
        blocks = hq.hq_fuse(30, circ.gates, kmax)
        assert len(blocks) < bound
        assert max(len(q) for q, _ in blocks) <= kmax


def test_fuse_errors(hq):
    lib = hq.load()
    circ = C.Circuit(4, [C.Gate("U", (0, 1, 2), np.eye(8, dtype=np.complex128))])
    with pytest.raises(hq.HQError, match="K_TOO_LARGE"):
        hq.hq_fuse(4, circ.gates, 2)
    with pytest.raises(hq.HQError, match="ARG"):
        hq.hq_fuse(4, circ.gates, 7)
    with pytest.raises(hq.HQError, match="ARG"):
        hq.hq_fuse(4, circ.gates, 3, method="dag", restarts=0)
    with pytest.raises(hq.HQError, match="K_TOO_LARGE"):
        hq.hq_fuse(4, circ.gates, 2, method="dag")
    # capacity: one slot for two disjoint-but-too-wide gates
    gates = (hq.hq_gate * 2)()
    keep = []
    for i, qs in enumerate([(0, 1), (2, 3)]):
        gates[i] = hq._gate_struct(qs, np.eye(4), keep)
    blocks = (hq.hq_gate * 1)()
    B = hq.ctypes.c_int(1)
    pool = np.zeros(64)
    rc = lib.hq_fuse(4, gates, 2, 2, blocks, hq.ctypes.byref(B), pool.ctypes.data_as(hq.ctypes.c_void_p), 64, None)
    assert rc == -11 and B.value == 2


def test_fuse_empty_circuit(hq):
    assert hq.hq_fuse(3, [], 4) == []
    assert hq.hq_fuse(3, [], 4, method="dag") == []


def test_batch_planner_host_only(hq):
    """hq_batch_workspace_bytes plans on the host (no device work): positive
    for a valid batch, 0 for invalid input."""
    cs = C.config_batch(8, seed=2, n_range=(3, 14), depth_range=(2, 6))
    assert hq.hq_batch_workspace_bytes(cs) > 0
    assert hq.hq_batch_workspace_bytes(cs, 13, 7) > 0
    assert hq.hq_batch_workspace_bytes(cs, 14, 6) == 0        # tile_bits out of range
    wide = C.Circuit(4, [C.Gate("U", (0, 1, 2), np.eye(8, dtype=np.complex128))])
    assert hq.hq_batch_workspace_bytes([wide]) == 0           # k > 2
