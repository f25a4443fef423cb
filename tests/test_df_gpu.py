"""complex128 gates in double-float arithmetic (HQ_ENGINE_DF: hi + lo float
pairs on the FP32 pipes) against the oracle at the complex128 bar,
max-abs 1e-12: dense gates k = 1..4 at every position class, monomial and
diagonal gates, whole circuits per gate and fused, magnitudes over many
octaves and non-unitary scaling."""
import math

import numpy as np
import pytest

import oracle
from paper_2111_06868_gb300 import circuits as C

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BAR = 1e-12


@pytest.fixture(scope="module")
def hq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_06868_gb300 import build
    from paper_2111_06868_gb300 import hq as _hq

    build.build()
    _hq.load()
    return _hq


def np_state(n, seed):
    rng = np.random.default_rng(seed)  # input only
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return psi / np.linalg.norm(psi)


def dev(psi):
    return torch.from_numpy(np.ascontiguousarray(psi, np.complex128)).cuda()


def max_abs(st, want):
    return float(np.abs(st.cpu().numpy() - want).max())


def qsets(n, k, seed):
    rng = C.SplitMix64(seed)
    rnd = []
    while len(rnd) < k:
        q = rng.randint(0, n - 1)
        if q not in rnd:
            rnd.append(q)
    return [list(range(n - k, n)), list(range(k)), rnd, [n - 1] + list(range(k - 1))]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [4, 11, 13, 20])
def test_dense_gates_every_position_class(hq, k, n):
    rng = C.SplitMix64(17 * n + k)
    psi = np_state(n, n + 3 * k)
    st = dev(psi)
    for qs in qsets(n, k, 5 * n + k):
        M = C.random_unitary(k, rng)
        hq.hq_apply_blocks(st, [(qs, M)], engine="df")
        oracle.apply_gate(psi, n, qs, M)
        assert max_abs(st, psi) <= BAR, qs


@pytest.mark.parametrize("n", [6, 15])
def test_monomial_and_diagonal_gates(hq, n):
    rng = C.SplitMix64(91 + n)
    psi = np_state(n, 7 + n)
    st = dev(psi)
    gates = [((0,), np.array([[0, 1], [1, 0]], complex)), ((n - 1, 1), C.cnot()), ((2, n - 2), C.swap()),
             ((3, 1), C.fsim(math.pi / 2, math.pi / 6)), ((1,), C.rot("Z", 0.7)), ((0, n - 1), C.cz()),
             ((4, 2, 0), np.diag(np.exp(1j * np.arange(8) * 0.37)))]
    # a random permutation with phases on 4 qubits, and a random diagonal on 6
    perm = [5, 3, 12, 0, 9, 14, 1, 7, 2, 11, 15, 4, 8, 6, 13, 10]
    P = np.zeros((16, 16), complex)
    for r, c in enumerate(perm):
        P[r, c] = np.exp(2j * math.pi * rng.uniform())
    gates.append(((1, 3, 0, 5), P))
    gates.append(((0, 1, 2, 3, 4, 5), np.diag(np.exp(2j * math.pi * np.array([rng.uniform() for _ in range(64)])))))
    for qs, M in gates:
        hq.hq_apply_blocks(st, [(qs, M)], engine="df")
        oracle.apply_gate(psi, n, qs, M)
        assert max_abs(st, psi) <= BAR, qs


@pytest.mark.parametrize("kmax", [1, 2, 3, 4])
def test_grid_circuit_per_gate_and_fused(hq, kmax):
    """n = 12 random circuit (163 gates) and an n = 16 fSim circuit, from
    |0..0>, per gate (kmax = 1) or fused into blocks of at most kmax qubits."""
    for circ in (C.config_small(seed=1), C.random_circuit(C.grid(4, 4), 12, seed=4, two_qubit="fsim")):
        want = oracle.simulate(circ)
        st = torch.empty(1 << circ.n, dtype=torch.complex128, device="cuda")
        hq.hq_state_init(st)
        blocks = [(g.qubits, g.matrix) for g in circ.gates] if kmax == 1 else hq.hq_fuse(circ.n, circ.gates, kmax)
        hq.hq_apply_blocks(st, blocks, engine="df")
        err = max_abs(st, want)
        print(f"n={circ.n} G={len(circ.gates)} kmax={kmax}: max-abs {err:.2e}")
        assert err <= BAR


def test_circuit_and_inverse_return_to_zero(hq):
    """C then C^dagger on the n = 14 grid: |0..0> back to within the bar."""
    circ = C.random_circuit(C.grid(2, 7), 16, seed=6, two_qubit="fsim")
    blocks = hq.hq_fuse(circ.n, circ.gates, 4)
    st = torch.empty(1 << circ.n, dtype=torch.complex128, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, blocks, engine="df")
    hq.hq_apply_blocks(st, [(q, m.conj().T.copy()) for q, m in reversed(blocks)], engine="df")
    want = np.zeros(1 << circ.n, complex)
    want[0] = 1
    assert max_abs(st, want) <= BAR


@pytest.mark.parametrize("scale", [1e-3, 37.0])
def test_non_unitary_scaling(hq, scale):
    n, k = 12, 4
    rng = C.SplitMix64(3)
    M = scale * C.random_unitary(k, rng)
    psi = np_state(n, 2)
    st = dev(psi)
    qs = [2, 9, 4, 11]
    hq.hq_apply_blocks(st, [(qs, M)], engine="df")
    oracle.apply_gate(psi, n, qs, M)
    assert max_abs(st, psi) <= BAR * max(1.0, scale)


def test_magnitudes_over_many_octaves(hq):
    """Amplitudes from 2^-60 to 1 (and exact zeros, negative zeros): the
    split into hi + lo and the rebuild keep 48 bits of every one."""
    n = 12
    psi = np_state(n, 9)
    octave = np.array([-(i % 61) for i in range(1 << n)], float)
    psi = psi * np.exp2(octave)
    psi[::97] = 0.0
    psi[5::211] = -0.0
    psi /= np.linalg.norm(psi)
    st = dev(psi)
    for qs, M in (((3,), C.hadamard()), ((0, 7), C.random_unitary(2, C.SplitMix64(1))),
                  ((11, 2, 5), C.random_unitary(3, C.SplitMix64(2)))):
        hq.hq_apply_blocks(st, [(qs, M)], engine="df")
        oracle.apply_gate(psi, n, qs, M)
    got = st.cpu().numpy()
    assert np.abs(got - psi).max() <= BAR
    big = np.abs(psi) > 1e-6
    rel = np.abs(got[big] - psi[big]) / np.abs(psi[big])
    assert rel.max() <= 1e-10, rel.max()  # 24-bit pairs would show ~6e-8


def test_engine_rejects_complex64(hq):
    st = torch.zeros(1 << 5, dtype=torch.complex64, device="cuda")
    with pytest.raises(hq.HQError, match="DTYPE"):
        hq.hq_apply_blocks(st, [((0,), C.hadamard())], engine="df")


@pytest.mark.slow
def test_n28_subset_fused_against_oracle(hq, n28_oracle):
    """The 28-qubit subset of the 33-qubit layout (942 gates) fused into
    blocks of at most 4 qubits, in double-float, against the oracle."""
    circ, want = n28_oracle
    st = torch.empty(1 << 28, dtype=torch.complex128, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, hq.hq_fuse(28, circ.gates, 4, method="dag"), engine="df")
    got = st.cpu().numpy()
    del st
    torch.cuda.empty_cache()
    err = float(np.abs(got - want).max())
    print(f"n=28 subset fused k<=4 double-float: max-abs {err:.2e}")
    assert err <= BAR
