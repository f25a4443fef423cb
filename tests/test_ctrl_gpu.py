"""Controlled-gate kernel (k_ctrl): CNOT, CZ, CPHASE, Toffoli and controlled
dense U with controls and targets anywhere, against the oracle.  Only the
amplitudes whose controls are all 1 may change."""
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


def controlled(U, nc):
    """nc controls (local MSBs) on U, built as P1..P1 (x) U + (I - P1..P1 (x) I)."""
    kt = int(U.shape[0]).bit_length() - 1
    on = np.ones((1, 1), np.complex128)
    for _ in range(nc):
        on = np.kron(on, np.diag([0, 1]).astype(np.complex128))
    return np.kron(on, U) + np.eye(1 << (nc + kt), dtype=np.complex128) - np.kron(on, np.eye(1 << kt))


def gate_list(n):
    """(qubits, matrix) with controls on high, middle and the lowest bits and
    targets anywhere; qubit q is flat bit n-1-q."""
    rng = C.SplitMix64(n)
    hi, lo = 0, n - 1
    out = [((hi, lo), C.cnot()), ((lo, hi), C.cnot()), ((n - 3, 2), C.cnot()), ((n - 1, 5), C.cnot()),
           ((n - 2, n - 1), C.cnot()), ((3, 7), C.cz()), ((n - 1, n - 2), C.cz()), ((1, n - 3), C.cphase(0.37)),
           ((n - 1, 4), C.cphase(-1.1)), ((0, 5, n - 1), controlled(C.PAULI["X"], 2)),
           ((n - 1, n - 2, 2), controlled(C.PAULI["X"], 2)), ((4, 1, 6), controlled(C.cz(), 1))]
    for nc, kt in [(1, 1), (1, 2), (2, 2), (3, 1), (4, 2), (2, 0), (5, 0)]:
        U = C.random_unitary(kt, rng) if kt else np.array([[np.exp(0.9j)]])
        qs = []
        while len(qs) < nc + kt:
            q = rng.randint(0, n - 1)
            if q not in qs:
                qs.append(q)
        out.append((tuple(qs), controlled(U, nc)))
    return out


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
@pytest.mark.parametrize("n", [14, 19])
def test_controlled_gates_match_oracle(hq, dtype, n):
    psi = random_state(n, 3 * n)
    st = torch.from_numpy(psi).to(getattr(torch, dtype)).cuda()
    for qs, M in gate_list(n):
        before = st.clone()
        hq.hq_apply_gate(st, qs, M)
        oracle.apply_gate(psi, n, qs, M)
        # amplitudes with some control 0 are untouched
        _, mask, _ = hq.hq_gate_structure(M)
        idx = np.arange(1 << n)
        on = np.ones(1 << n, bool)
        for j, q in enumerate(qs):
            if (mask >> j) & 1:
                on &= ((idx >> (n - 1 - q)) & 1) == 1
        off = torch.from_numpy(~on).cuda()
        assert torch.equal(st[off], before[off]), qs
    got = st.cpu().numpy().astype(np.complex128)
    if dtype == "complex128":
        assert np.abs(got - psi).max() <= 1e-12
    else:
        assert np.linalg.norm(got - psi) / np.linalg.norm(psi) <= 2e-6


@pytest.mark.parametrize("engine", ["auto", "tc_f16"])
def test_controlled_blocks_in_block_lists(hq, engine):
    """hq_apply_blocks routes controlled blocks (here up to 6 qubits, which the
    tensor-core engine would otherwise take) to the controlled kernel."""
    n = 18
    psi = random_state(n, 5)
    st = torch.from_numpy(psi).to(torch.complex64).cuda()
    blocks = gate_list(n)
    hq.hq_apply_blocks(st, blocks, engine=engine, tc_min_k=4)
    for qs, M in blocks:
        oracle.apply_gate(psi, n, qs, M)
    got = st.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - psi) / np.linalg.norm(psi) <= 4e-6


def test_qft_and_ghz_through_controlled_kernel(hq):
    """Circuits made of controlled gates: GHZ (H + CNOT chain) in complex128
    gives 1/sqrt(2) at 0 and 2^n - 1; the QFT matches the oracle."""
    n = 16
    ghz = [((0,), C.hadamard())] + [((q, q + 1), C.cnot()) for q in range(n - 1)]
    st = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, ghz)
    got = st.cpu().numpy()
    want = np.zeros(1 << n, np.complex128)
    want[0] = want[-1] = 2 ** -0.5
    assert np.abs(got - want).max() <= 1e-14
    circ = C.Circuit(n, C.basis_prep(n, 12345).gates + C.qft_circuit(n).gates)
    st = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, [(g.qubits, g.matrix) for g in circ.gates])
    assert np.abs(st.cpu().numpy() - oracle.simulate(circ)).max() <= 1e-12
