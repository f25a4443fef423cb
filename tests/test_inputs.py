"""The seeded synthetic workloads: gate counts, edge patterns, gate
definitions.  Host only."""
import math

import numpy as np
import pytest

from paper_2111_06868_gb300 import circuits as C


def test_splitmix64_reference_values():
    # first outputs for seed 0 of the published SplitMix64 definition
    r = C.SplitMix64(0)
    assert r.next_u64() == 0xE220A8397B1DCDAF
    assert r.next_u64() == 0x6E789E6AA1B965F4


@pytest.mark.parametrize("name,f,P", [("X", C.sqrt_x, "X"), ("Y", C.sqrt_y, "Y")])
def test_sqrt_paulis_square(name, f, P):
    m = f()
    np.testing.assert_allclose(m @ m, -1j * C.PAULI[P], atol=1e-15)
    np.testing.assert_allclose(m @ m.conj().T, np.eye(2), atol=1e-15)


def test_sqrt_w_square():
    W = (C.PAULI["X"] + C.PAULI["Y"]) / math.sqrt(2)
    m = C.sqrt_w()
    np.testing.assert_allclose(m @ m, -1j * W, atol=1e-15)


def test_fsim_and_rotations_unitary():
    for m in [C.fsim(math.pi / 2, math.pi / 6), C.rot("X", 0.3), C.rot("Y", 1.1), C.rot("Z", 2.9), C.cz()]:
        np.testing.assert_allclose(m @ m.conj().T, np.eye(m.shape[0]), atol=1e-15)
    # R_Z(t) = diag(e^{-it/2}, e^{it/2})
    np.testing.assert_allclose(np.diag(C.rot("Z", 0.4)), [np.exp(-0.2j), np.exp(0.2j)], atol=1e-15)


def counts(circ):
    one = sum(1 for g in circ.gates if g.k == 1)
    two = sum(1 for g in circ.gates if g.k == 2)
    return one, two


def test_config_small_counts():
    c = C.config_small(0)
    assert c.n == 12 and counts(c) == (120, 43)


def test_config_n30_counts():
    c = C.config_n30(0)
    assert c.n == 30 and counts(c) == (600, 245)
    g = C.grid(5, 6)
    assert [len(g.pattern(p)) for p in range(4)] == [15, 10, 12, 12]


def test_config_n33_counts_and_subset():
    c = C.config_n33(0)
    assert c.n == 33 and counts(c) == (792, 324)
    g = C.grid(**C.SITES_33)
    assert [len(g.pattern(p)) for p in range(4)] == [15, 12, 15, 12]
    s = C.config_n33(0, first=28)
    assert s.n == 28
    assert all(max(gt.qubits) < 28 for gt in s.gates)


def test_never_same_gate_twice():
    c = C.config_n30(1)
    last = {}
    for g in c.gates:
        if g.k == 1:
            q = g.qubits[0]
            assert last.get(q) != g.name
            last[q] = g.name


def test_ansatz_shape():
    c = C.ansatz(20, 8)
    assert c.n_params == 320
    assert sum(1 for g in c.gates if g.axis) == 320
    assert sum(1 for g in c.gates if g.name == "CZ") == 152
    H = C.ansatz_hamiltonian(20)
    assert len(H) == 39
    th = C.ansatz_params(320, 2, 0)
    assert th.shape == (2, 320) and th.min() >= 0 and th.max() < 2 * math.pi


def test_batch_config_ranges():
    cs = C.config_batch(24, seed=1)
    assert all(10 <= c.n <= 24 for c in cs)
    for c in cs:
        assert all(max(g.qubits) < c.n for g in c.gates)


def test_seeded_determinism():
    a, b = C.config_n30(5), C.config_n30(5)
    assert [g.name for g in a.gates] == [g.name for g in b.gates]
    assert [g.name for g in a.gates] != [g.name for g in C.config_n30(6).gates]
