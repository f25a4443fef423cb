"""Monomial gates (one nonzero per row and column: X, Y, CNOT, SWAP, iSWAP,
Toffoli, fSim(pi/2, phi), random permutations with random phases) take the
permute-and-phase kernel; results against the oracle's dense application."""
import cmath
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


def random_state(n, seed):
    rng = np.random.default_rng(seed)  # input only
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return psi / np.linalg.norm(psi)


def random_monomial(k, rng):
    d = 1 << k
    perm = list(range(d))
    for i in range(d - 1, 0, -1):  # seeded shuffle
        j = rng.randint(0, i)
        perm[i], perm[j] = perm[j], perm[i]
    m = np.zeros((d, d), np.complex128)
    for r in range(d):
        m[r, perm[r]] = cmath.exp(1j * 2 * math.pi * rng.uniform())
    return m


X = np.array([[0, 1], [1, 0]], complex)
Y = np.array([[0, -1j], [1j, 0]], complex)
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], complex)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], complex)
ISWAP = np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]], complex)
TOFFOLI = np.eye(8, dtype=complex)[[0, 1, 2, 3, 4, 5, 7, 6]]
NAMED = [(X, 1), (Y, 1), (CNOT, 2), (SWAP, 2), (ISWAP, 2), (C.fsim(math.pi / 2, math.pi / 6), 2), (TOFFOLI, 3)]


@pytest.mark.parametrize("dt,tol", [(torch.complex64, 2e-6), (torch.complex128, 1e-12)])
@pytest.mark.parametrize("n", [3, 9, 14])
def test_named_and_random_monomials_every_position(hq, dt, tol, n):
    rng = C.SplitMix64(13 * n)
    psi = random_state(n, n)
    st = torch.from_numpy(psi).to(dt).cuda()
    gates = list(NAMED) + [(random_monomial(k, rng), k) for k in (1, 2, 3, 4) for _ in range(2)]
    for m, k in gates:
        if k > n:
            continue
        for qs in ([n - 1 - j for j in range(k)], list(range(k)), [(3 * j + 1) % n for j in range(k)] if n >= 3 * k else list(range(k))):
            if len(set(qs)) < k:
                continue
            hq.hq_apply_gate(st, qs, m)
            oracle.apply_gate(psi, n, qs, m)
    got = st.cpu().numpy().astype(np.complex128)
    if dt == torch.complex128:
        assert np.max(np.abs(got - psi)) <= tol
    else:
        assert np.linalg.norm(got - psi) / np.linalg.norm(psi) <= tol * 50


def test_fsim_circuit_through_apply_blocks(hq):
    """The n=16 grid circuit unfused (fSim(pi/2, pi/6) is monomial) in both precisions."""
    circ = C.random_circuit(C.layout_for(16), 8, seed=4, two_qubit="fsim")
    want = oracle.simulate(circ)
    for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 2e-5)):
        st = torch.empty(1 << 16, dtype=dt, device="cuda")
        hq.hq_state_init(st)
        hq.hq_apply_blocks(st, [(g.qubits, g.matrix) for g in circ.gates])
        got = st.cpu().numpy().astype(np.complex128)
        err = np.max(np.abs(got - want)) if dt == torch.complex128 else np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err <= tol, (dt, err)
