"""Circuit utilities ahead of fusion (Sec. 3.1): simplify() and pop(), host
only.  Pinned by the paper's own simplify example and by invariants the
oracle checks: the kept gates give the same state (simplify) or the same
reduced state on the pinned qubits (pop)."""
import numpy as np
import pytest

import oracle
from paper_2111_06868_gb300 import circuits as C


@pytest.fixture(scope="module")
def hq():
    from paper_2111_06868_gb300 import build
    from paper_2111_06868_gb300 import hq as _hq

    build.build()
    _hq.load()
    return _hq


def shuffled(items, seed):
    items = list(items)
    r = C.SplitMix64(seed)
    for i in range(len(items) - 1, 0, -1):
        j = r.randint(0, i)
        items[i], items[j] = items[j], items[i]
    return items


def dagger(g):
    return C.Gate(g.name + "^dag", g.qubits, g.matrix.conj().T)


def test_paper_simplify_example(hq):
    """Sec. 3.1: CPHASE on all pairs of 5 qubits followed by the inverse of a
    shuffled copy simplifies to the empty circuit when commutation through
    the gates' matrices is used (all CPHASEs commute)."""
    circ = [C.Gate("CPHASE", (a, b), C.cphase(1.0)) for a in range(5) for b in range(a + 1, 5)]
    inv = [dagger(g) for g in shuffled(circ, 0)][::-1]
    assert hq.hq_simplify(5, circ + inv) == []
    # without matrix commutation nothing meets its inverse here, and what is
    # kept is still the same operator
    kept = hq.hq_simplify(5, circ + inv, use_matrix_commutation=False)
    assert len(kept) == 20
    psi0 = oracle.state_init(5, "+-+-+")
    np.testing.assert_allclose(oracle.apply_circuit(psi0.copy(), C.Circuit(5, kept)), psi0, atol=1e-13)


def test_circuit_times_its_exact_inverse_is_empty_without_commutation(hq):
    circ = C.random_circuit(C.grid(2, 4), 6, seed=4, two_qubit="fsim").gates
    inv = [dagger(g) for g in circ][::-1]
    assert hq.hq_simplify(8, circ + inv, use_matrix_commutation=False) == []


@pytest.mark.parametrize("seed", range(4))
def test_simplify_keeps_the_operator(hq, seed):
    """A random circuit with cancelling pairs U, U^dag planted around a gate
    on other qubits: the planted pairs go, and the state is the oracle's of
    the full circuit."""
    n = 7
    rng = C.SplitMix64(100 + seed)
    gates = list(C.random_dense_circuit(n, 30, seed=seed, kmax=2).gates)
    planted = 0
    for _ in range(6):
        pos = rng.randint(0, len(gates))
        a, b = rng.randint(0, n - 1), rng.randint(0, n - 1)
        if a == b:
            continue
        U = C.random_unitary(2, rng)
        # U, then gates on other qubits and a diagonal phase on a, then U^dag
        others = [q for q in range(n) if q not in (a, b)]
        mid = [C.Gate("U1", (others[rng.randint(0, len(others) - 1)],), C.random_unitary(1, rng))]
        block = [C.Gate("U", (a, b), U)] + mid + [C.Gate("Udag", (a, b), U.conj().T)]
        gates[pos:pos] = block
        planted += 1
    kept = hq.hq_simplify(n, gates)
    assert len(kept) <= len(gates) - 2 * planted
    psi0 = oracle.state_init(n, "+-01+-0")
    np.testing.assert_allclose(oracle.apply_circuit(psi0.copy(), C.Circuit(n, kept)),
                               oracle.apply_circuit(psi0.copy(), C.Circuit(n, gates)), atol=1e-12)


def test_simplify_commutation_cases(hq):
    n = 3
    X = C.PAULI["X"]
    cn01, cn10 = C.Gate("CX", (0, 1), C.cnot()), C.Gate("CX", (1, 0), C.cnot())
    # the same qubit set in the other order is a different operator
    assert len(hq.hq_simplify(n, [cn01, cn10])) == 2
    assert hq.hq_simplify(n, [cn01, cn01]) == []
    # CNOT(0,1) and X(1) commute (X on the target): the pair cancels through it
    x1 = C.Gate("X", (1,), X)
    assert hq.hq_simplify(n, [cn01, x1, cn01]) == [x1]
    assert len(hq.hq_simplify(n, [cn01, x1, cn01], use_matrix_commutation=False)) == 3
    # X(0) on the control does not commute: nothing cancels
    x0 = C.Gate("X", (0,), X)
    assert len(hq.hq_simplify(n, [cn01, x0, cn01])) == 3
    # identities go, near-identities within atol go, larger deviations stay
    eye = C.Gate("I", (2,), np.eye(2, dtype=np.complex128))
    near = C.Gate("I~", (2,), np.eye(2, dtype=np.complex128) + 1e-14)
    far = C.Gate("I~~", (2,), np.eye(2, dtype=np.complex128) + 1e-9)
    assert hq.hq_simplify(n, [eye, near, far]) == [far]


def reduced(psi, n, keep):
    """Reduced density matrix of the qubits `keep` (ascending)."""
    t = psi.reshape((2,) * n)
    rest = [q for q in range(n) if q not in keep]
    t = np.moveaxis(t, keep + rest, list(range(n))).reshape(1 << len(keep), -1)
    return t @ t.conj().T


@pytest.mark.parametrize("pinned", [[0], [5], [1, 6], [3, 4, 7]])
def test_pop_right_keeps_the_pinned_reduced_state(hq, pinned):
    n = 8
    circ = C.random_circuit(C.grid(2, 4), 8, seed=sum(pinned), two_qubit="fsim").gates
    kept = hq.hq_pop(n, circ, pinned)
    assert len(kept) < len(circ)
    tokens = "+-01+-0+"
    full = oracle.simulate(C.Circuit(n, circ), tokens)
    part = oracle.simulate(C.Circuit(n, kept), tokens)
    np.testing.assert_allclose(reduced(part, n, sorted(pinned)), reduced(full, n, sorted(pinned)), atol=1e-12)
    H = [(1.0, ((pinned[0], "Z"),)), (0.5, ((pinned[-1], "X"),))]
    assert abs(oracle.expectation(part, H) - oracle.expectation(full, H)) <= 1e-12


def test_pop_light_cone_by_hand(hq):
    """A chain: CNOT(0,1), CNOT(1,2), CNOT(2,3), then X on 3.  Pinned {1}
    from the right keeps the first two (qubit 1's cone at the output); pinned
    {3} keeps all; from the left, pinned {3} keeps only the last two and
    pinned {0} all four (the chain carries qubit 0's cone to qubit 3)."""
    X, cn = C.PAULI["X"], C.cnot()
    g = [C.Gate("CX", (0, 1), cn), C.Gate("CX", (1, 2), cn), C.Gate("CX", (2, 3), cn), C.Gate("X", (3,), X)]
    assert hq.hq_pop(4, g, [1]) == g[:2]
    assert hq.hq_pop(4, g, [3]) == g
    assert hq.hq_pop(4, g, [3], "left") == g[2:]
    assert hq.hq_pop(4, g, [0], "left") == g
    assert hq.hq_pop(4, g, []) == []


def test_pop_left_is_pop_right_of_the_inverse(hq):
    n = 8
    circ = C.random_circuit(C.grid(2, 4), 8, seed=9, two_qubit="fsim").gates
    left = hq.hq_pop(n, circ, [2, 5], "left")
    inv = [dagger(g) for g in circ][::-1]
    right_inv = hq.hq_pop(n, inv, [2, 5], "right")
    assert [g.qubits for g in left][::-1] == [g.qubits for g in right_inv]
    # the reduced state on {2, 5} after the inverse circuit is kept
    tokens = "0+1-0+1-"
    full = oracle.simulate(C.Circuit(n, inv), tokens)
    part = oracle.simulate(C.Circuit(n, [dagger(g) for g in left][::-1]), tokens)
    np.testing.assert_allclose(reduced(part, n, [2, 5]), reduced(full, n, [2, 5]), atol=1e-12)


def test_errors(hq):
    g = [C.Gate("X", (0,), C.PAULI["X"])]
    with pytest.raises(hq.HQError, match="QUBIT_RANGE"):
        hq.hq_pop(2, g, [2])
    with pytest.raises(hq.HQError, match="QUBIT_RANGE"):
        hq.hq_pop(1, [C.Gate("X", (1,), C.PAULI["X"])], [0])
    with pytest.raises(hq.HQError, match="ARG"):
        hq.hq_simplify(2, g, atol=-1.0)
    lib = hq.load()
    assert lib.hq_pop(2, None, 1, None, 0, 0, None) == -1
    assert lib.hq_simplify(2, None, 1, 1, 1e-12, None) == -1
    assert hq.hq_simplify(3, []) == [] and hq.hq_pop(3, [], [0]) == []
