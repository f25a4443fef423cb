"""Gate-structure detection (hq_gate_structure, host only): which gates the
controlled, diagonal and monomial kernels take.  Controlled gates (Sec. 2's
Control) are built here independently of the detector, as P0 (x) I + P1 (x) U
with np.kron and a transpose of the qubit axes, and the detector's split is
checked by rebuilding the matrix from it."""
import itertools

import numpy as np
import pytest

from paper_2111_06868_gb300 import circuits as C


@pytest.fixture(scope="module")
def hq():
    from paper_2111_06868_gb300 import build
    from paper_2111_06868_gb300 import hq as _hq

    build.build()
    _hq.load()
    return _hq


P0 = np.diag([1, 0]).astype(np.complex128)
P1 = np.diag([0, 1]).astype(np.complex128)


def controlled(U, nc):
    """nc controls first (local MSBs), then U's qubits: the projector onto
    'all controls 1' times U, plus the identity on the rest."""
    kt = int(U.shape[0]).bit_length() - 1
    on = np.ones((1,), np.complex128).reshape(1, 1)
    for _ in range(nc):
        on = np.kron(on, P1)
    full = np.kron(on, U)
    rest = np.eye(1 << (nc + kt), dtype=np.complex128) - np.kron(on, np.eye(1 << kt))
    return full + rest


def permute_qubits(M, order):
    """The same operator with its qubits listed in `order` (new position i
    holds old qubit order[i])."""
    k = int(M.shape[0]).bit_length() - 1
    T = M.reshape((2,) * (2 * k))
    T = T.transpose(list(order) + [k + o for o in order])
    return T.reshape(1 << k, 1 << k)


def rebuild(k, mask, u):
    """Matrix from a control mask and the target block, entry by entry."""
    ctrl = [j for j in range(k) if (mask >> j) & 1]
    targ = [j for j in range(k) if not (mask >> j) & 1]
    M = np.eye(1 << k, dtype=np.complex128)
    for r in range(1 << k):
        for c in range(1 << k):
            bits_r = [(r >> (k - 1 - j)) & 1 for j in range(k)]
            bits_c = [(c >> (k - 1 - j)) & 1 for j in range(k)]
            if all(bits_r[j] for j in ctrl) and all(bits_c[j] for j in ctrl):
                a = int("".join(str(bits_r[j]) for j in targ) or "0", 2)
                b = int("".join(str(bits_c[j]) for j in targ) or "0", 2)
                M[r, c] = u[a, b]
    return M


def test_named_gates(hq):
    D, Mo, Ct = hq.STRUCT_DIAGONAL, hq.STRUCT_MONOMIAL, hq.STRUCT_CONTROLLED
    s, m, u = hq.hq_gate_structure(C.cnot())
    assert (s, m) == (Mo | Ct, 0b01) and np.array_equal(u, C.PAULI["X"])
    s, m, u = hq.hq_gate_structure(C.cz())
    assert (s, m) == (D | Mo | Ct, 0b11) and u.shape == (1, 1) and u[0, 0] == -1
    s, m, u = hq.hq_gate_structure(C.cphase(0.7))
    assert (s, m) == (D | Mo | Ct, 0b11) and np.isclose(u[0, 0], np.exp(0.7j))
    tof = controlled(C.PAULI["X"], 2)
    s, m, u = hq.hq_gate_structure(tof)
    assert (s, m) == (Mo | Ct, 0b011) and np.array_equal(u, C.PAULI["X"])
    for M in (C.hadamard(), C.swap(), C.fsim(np.pi / 2, np.pi / 6), C.sqrt_x(), C.random_unitary(2, C.SplitMix64(3))):
        s, m, _ = hq.hq_gate_structure(M)
        assert not s & Ct and m == 0, M
    assert hq.hq_gate_structure(C.swap())[0] == Mo
    assert hq.hq_gate_structure(C.fsim(np.pi / 2, np.pi / 6))[0] == Mo
    assert hq.hq_gate_structure(C.random_unitary(3, C.SplitMix64(4)))[0] == 0
    # the identity: every qubit is a control of a 1x1 identity
    s, m, u = hq.hq_gate_structure(np.eye(8, dtype=np.complex128))
    assert m == 0b111 and u.shape == (1, 1) and u[0, 0] == 1


@pytest.mark.parametrize("nc,kt", [(1, 1), (1, 2), (2, 1), (2, 2), (3, 1), (1, 3), (4, 2)])
def test_controlled_in_any_qubit_order(hq, nc, kt):
    rng = C.SplitMix64(10 * nc + kt)
    U = C.random_unitary(kt, rng)
    base = controlled(U, nc)
    k = nc + kt
    for perm_seed in range(3):
        order = list(range(k))
        r = C.SplitMix64(perm_seed)
        for i in range(k - 1, 0, -1):
            j = r.randint(0, i)
            order[i], order[j] = order[j], order[i]
        M = permute_qubits(base, order)
        s, mask, u = hq.hq_gate_structure(M)
        want_mask = sum(1 << i for i, o in enumerate(order) if o < nc)
        assert s & hq.STRUCT_CONTROLLED and mask == want_mask, (order, mask)
        np.testing.assert_allclose(rebuild(k, mask, u), M, atol=1e-15)
        # U appears with its qubits in their new relative order
        targ_order = [o - nc for o in order if o >= nc]
        np.testing.assert_allclose(u, permute_qubits(U, targ_order), atol=1e-15)


def test_near_identity_entries_within_tolerance(hq):
    """Entries within 4 FP64 epsilon of the identity count as exact (as the
    monomial test treats tiny entries as zero); larger ones do not."""
    M = C.cnot().copy()
    M[0, 1] = 1e-17
    assert hq.hq_gate_structure(M)[1] == 0b01
    M[0, 1] = 1e-12
    assert hq.hq_gate_structure(M)[1] == 0


def test_every_two_qubit_permutation_matrix(hq):
    """Brute force over the 24 permutations of a 2-qubit basis: a qubit is a
    control exactly when the permutation fixes every state with that qubit 0."""
    for p in itertools.permutations(range(4)):
        M = np.zeros((4, 4), np.complex128)
        for c, r in enumerate(p):
            M[r, c] = 1
        _, mask, _ = hq.hq_gate_structure(M)
        want = 0
        for j in range(2):
            bit = 1 << (1 - j)
            if all(p[x] == x for x in range(4) if not x & bit):
                want |= 1 << j
        assert mask == want, (p, mask)


def test_errors(hq):
    lib = hq.load()
    assert lib.hq_gate_structure(2, None, None, None) == -1
    m = np.eye(2, dtype=np.complex128)
    assert lib.hq_gate_structure(0, m.ctypes.data_as(hq.ctypes.c_void_p), None, None) == -4
    assert lib.hq_gate_structure(7, m.ctypes.data_as(hq.ctypes.c_void_p), None, None) == -4
    assert lib.hq_gate_structure(1, m.ctypes.data_as(hq.ctypes.c_void_p), None, None) == (
        hq.STRUCT_DIAGONAL | hq.STRUCT_MONOMIAL | hq.STRUCT_CONTROLLED)
