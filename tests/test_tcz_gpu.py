"""complex128 blocks on the tensor cores (HQ_ENGINE_TC_C128: exact FP16
products of 8-bit signed digit slices, FP32 accumulation exact, levels joined
in 64-bit integers) against the oracle at the complex128 bar, max-abs 1e-12:
single dense 4- and 3-qubit blocks at every position class, whole circuits
fused into blocks of at most 3 and 4 qubits, magnitudes over many octaves,
non-unitary scaling, zero groups, the 28-qubit subset, and allocation
failure."""
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
    # high targets (short runs), low targets (one run), random order, split
    return [list(range(n - k, n)), list(range(k)), rnd, [n - 1] + list(range(k - 1))[::-1]]


@pytest.mark.parametrize("k", [3, 4])
@pytest.mark.parametrize("n", [11, 12, 14, 19])
def test_single_block_every_position_class(hq, k, n):
    rng = C.SplitMix64(29 * n + k)
    psi = np_state(n, 3 * n + k)
    st = dev(psi)
    for qs in qsets(n, k, 11 * n + k):
        M = C.random_unitary(k, rng)
        hq.hq_apply_blocks(st, [(qs, M)], engine="tc_c128")
        oracle.apply_gate(psi, n, qs, M)
        err = max_abs(st, psi)
        assert err <= BAR, (qs, err)


@pytest.mark.parametrize("kmax", [3, 4])
def test_grid_circuits_fused(hq, kmax):
    """The n = 12 random circuit (163 gates) and an n = 16 fSim circuit from
    |0..0>, fused into blocks of at most kmax qubits: dense blocks on the
    tensor cores, the others in double-float."""
    for circ in (C.config_small(seed=1), C.random_circuit(C.grid(4, 4), 12, seed=4, two_qubit="fsim")):
        want = oracle.simulate(circ)
        st = torch.empty(1 << circ.n, dtype=torch.complex128, device="cuda")
        hq.hq_state_init(st)
        hq.hq_apply_blocks(st, hq.hq_fuse(circ.n, circ.gates, kmax, method="beam", width=32), engine="tc_c128")
        err = max_abs(st, want)
        print(f"n={circ.n} G={len(circ.gates)} kmax={kmax}: max-abs {err:.2e}")
        assert err <= BAR


def test_circuit_and_inverse_return_to_zero(hq):
    circ = C.random_circuit(C.grid(2, 7), 16, seed=6, two_qubit="fsim")
    blocks = hq.hq_fuse(circ.n, circ.gates, 4, method="beam", width=32)
    st = torch.empty(1 << circ.n, dtype=torch.complex128, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, blocks, engine="tc_c128")
    hq.hq_apply_blocks(st, [(q, m.conj().T.copy()) for q, m in reversed(blocks)], engine="tc_c128")
    want = np.zeros(1 << circ.n, complex)
    want[0] = 1
    assert max_abs(st, want) <= BAR


@pytest.mark.parametrize("scale", [1e-3, 37.0, 2.0 ** 70])
def test_non_unitary_scaling(hq, scale):
    n, k = 12, 4
    M = scale * C.random_unitary(k, C.SplitMix64(3))
    psi = np_state(n, 2)
    st = dev(psi)
    qs = [2, 9, 4, 11]
    hq.hq_apply_blocks(st, [(qs, M)], engine="tc_c128")
    oracle.apply_gate(psi, n, qs, M)
    assert max_abs(st, psi) <= BAR * max(1.0, scale)


def test_magnitudes_over_many_octaves_and_zero_groups(hq):
    """Amplitudes from 2^-60 to 1, exact and negative zeros, whole groups of
    zeros: every group is scaled by its own largest exponent, so the error
    stays below 1e-10 of the state's largest amplitude, and amplitudes near
    the top keep ~35 bits."""
    n = 13
    psi = np_state(n, 9)
    psi = psi * np.exp2(np.array([-(i % 61) for i in range(1 << n)], float))
    psi[::97] = 0.0
    psi[5::211] = -0.0
    psi[: 1 << 5] = 0.0  # targets 0..3 below: the first groups are all zero
    psi /= np.linalg.norm(psi)
    st = dev(psi)
    for qs in ((9, 10, 11, 12), (0, 5, 7, 12), (3, 1, 8)):
        M = C.random_unitary(len(qs), C.SplitMix64(len(qs) + qs[0]))
        hq.hq_apply_blocks(st, [(qs, M)], engine="tc_c128")
        oracle.apply_gate(psi, n, qs, M)
    got = st.cpu().numpy()
    assert np.abs(got - psi).max() <= 1e-10 * np.abs(psi).max()
    big = np.abs(psi) > 1e-2 * np.abs(psi).max()
    assert (np.abs(got[big] - psi[big]) / np.abs(psi[big])).max() <= 1e-9


def test_structured_gates_take_the_double_float_kernels(hq):
    """Diagonal, monomial and small gates are not tensor-core blocks: with
    this engine they run as HQ_ENGINE_DF does (bit-equal)."""
    n = 12
    psi = np_state(n, 4)
    a, b = dev(psi), dev(psi)
    gates = [((0, 1, 2, 3), np.diag(np.exp(1j * np.arange(16) * 0.3))), ((4, 7), C.fsim(np.pi / 2, np.pi / 6)),
             ((2,), C.hadamard()), ((5, 9), C.random_unitary(2, C.SplitMix64(8)))]
    hq.hq_apply_blocks(a, gates, engine="tc_c128")
    hq.hq_apply_blocks(b, gates, engine="df")
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_engine_rejects_complex64(hq):
    st = torch.zeros(1 << 12, dtype=torch.complex64, device="cuda")
    with pytest.raises(hq.HQError, match="DTYPE"):
        hq.hq_apply_blocks(st, [((0, 1, 2, 3), C.random_unitary(4, C.SplitMix64(1)))], engine="tc_c128")


def test_allocation_failure_leaves_state(hq):
    n = 12
    psi = np_state(n, 6)
    st = dev(psi)
    M = C.random_unitary(4, C.SplitMix64(5))
    hq.hq_test_fail_next_allocs(1)
    try:
        with pytest.raises(hq.HQError, match="ALLOC"):
            hq.hq_apply_blocks(st, [((0, 3, 6, 9), M)], engine="tc_c128")
    finally:
        hq.hq_test_fail_next_allocs(0)
    assert max_abs(st, psi) == 0.0
    hq.hq_apply_blocks(st, [((0, 3, 6, 9), M)], engine="tc_c128")
    oracle.apply_gate(psi, n, (0, 3, 6, 9), M)
    assert max_abs(st, psi) <= BAR


@pytest.mark.slow
def test_n28_subset_fused_against_oracle(hq, n28_oracle):
    """The 28-qubit subset of the 33-qubit layout (942 gates) fused into
    blocks of at most 4 qubits on the tensor cores, against the oracle."""
    circ, want = n28_oracle
    st = torch.empty(1 << 28, dtype=torch.complex128, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, hq.hq_fuse(28, circ.gates, 4, method="beam", width=64), engine="tc_c128")
    got = st.cpu().numpy()
    del st
    torch.cuda.empty_cache()
    err = float(np.abs(got - want).max())
    print(f"n=28 subset fused k<=4 tensor-core complex128: max-abs {err:.2e}")
    assert err <= BAR
