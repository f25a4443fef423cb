"""Tensor-core engine (tcgen05, split FP16/BF16 products, FP32 accumulate) for
fused k = 5, 6 blocks, against the oracle.  FP16 hi+lo must meet the complex64
bar (relative L2 <= 2e-5 per 1000 unfused gates); BF16 hi+lo has ~16
significant bits and only its measured error is checked against a loose
bound."""
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


def rel_l2(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


def qsets(n, k, seed):
    rng = C.SplitMix64(seed)
    rnd = []
    while len(rnd) < k:
        q = rng.randint(0, n - 1)
        if q not in rnd:
            rnd.append(q)
    return [list(range(n - k, n)), list(range(k)), rnd, [n - 1, 0] + list(range(1, k - 1))[::-1]]


@pytest.mark.parametrize("engine,tol", [("tc_f16", 2e-6), ("tc_bf16", 3e-4)])
@pytest.mark.parametrize("k", [4, 5, 6])
@pytest.mark.parametrize("n", [11, 12, 13, 16, 20])
def test_single_block_every_position_class(hq, engine, tol, k, n):
    """n >= 13: k = 4, 5 blocks run widened to 6 qubits; n = 11, 12 keep the
    4- and 5-qubit kernels."""
    if n < k + 7:
        pytest.skip()
    rng = C.SplitMix64(31 * n + k)
    psi = random_state(n, n + k)
    st = torch.from_numpy(psi).to(torch.complex64).cuda()
    for qs in qsets(n, k, 7 * n + k):
        M = C.random_unitary(k, rng)
        hq.hq_apply_blocks(st, [(qs, M)], engine=engine, tc_min_k=4)
        oracle.apply_gate(psi, n, qs, M)
        err = rel_l2(st.cpu().numpy().astype(np.complex128), psi)
        assert err <= tol, (qs, err)


LOW_BIT_PATTERNS = [[0, 1, 2, 3, 4, 5], [1, 2, 3, 4, 7, 8], [0, 1, 6, 7, 12, 13], [2, 3, 4, 8, 9, 10],
                    [0, 2, 4, 6, 8, 10], [3, 4, 5, 9, 10, 11]]


@pytest.mark.parametrize("engine,tol", [("tc_f16", 2e-6), ("tc_bf16", 3e-4)])
@pytest.mark.parametrize("k", [4, 5, 6])
@pytest.mark.parametrize("pattern", range(len(LOW_BIT_PATTERNS)))
def test_low_bit_targets_in_any_order(hq, engine, tol, k, pattern):
    """Targets on the lowest flat bits (the four-threads-per-group mapping,
    with and without adjacent amplitude pairs), given in shuffled order."""
    n = 18
    bits = LOW_BIT_PATTERNS[pattern][:k]
    rng = C.SplitMix64(97 * k + pattern)
    qs = [n - 1 - b for b in bits]
    for i in range(len(qs) - 1, 0, -1):  # seeded shuffle of the target order
        j = rng.randint(0, i)
        qs[i], qs[j] = qs[j], qs[i]
    psi = random_state(n, 5 * k + pattern)
    st = torch.from_numpy(psi).to(torch.complex64).cuda()
    for _ in range(2):
        M = C.random_unitary(k, rng)
        hq.hq_apply_blocks(st, [(qs, M)], engine=engine, tc_min_k=4)
        oracle.apply_gate(psi, n, qs, M)
    err = rel_l2(st.cpu().numpy().astype(np.complex128), psi)
    assert err <= tol, (qs, err)


# Targets that leave a 9-bit contiguous run (2^9 amplitudes) at the bottom of
# the tile: tensor-map boxes whose rows take two dimensions, with 1-4 groups of
# high targets (the last one also loaded as two boxes).
SPLIT_ROW_PATTERNS = [[4, 5, 10, 11, 17, 23], [7, 8, 13, 14, 15, 20], [4, 5, 10, 11, 16, 17],
                      [7, 8, 12, 14, 16, 18], [0, 1, 11, 13, 15, 17]]


@pytest.mark.parametrize("pattern", range(len(SPLIT_ROW_PATTERNS)))
def test_nine_bit_runs_as_two_dimensional_box_rows(hq, pattern):
    n, k = 24, 6
    bits = SPLIT_ROW_PATTERNS[pattern]
    qs = [n - 1 - b for b in bits]
    rng = C.SplitMix64(211 + pattern)
    psi = random_state(n, 19 + pattern)
    st = torch.from_numpy(psi).to(torch.complex64).cuda()
    for _ in range(2):
        M = C.random_unitary(k, rng)
        hq.hq_apply_blocks(st, [(qs, M)], engine="tc_f16")
        oracle.apply_gate(psi, n, qs, M)
    err = rel_l2(st.cpu().numpy().astype(np.complex128), psi)
    assert err <= 2e-6, (bits, err)


@pytest.mark.parametrize("scale", [1e-3, 37.0])
def test_non_unitary_scaling(hq, scale):
    n, k = 14, 6
    rng = C.SplitMix64(5)
    M = scale * C.random_unitary(k, rng)
    psi = random_state(n, 3)
    st = torch.from_numpy(psi).to(torch.complex64).cuda()
    qs = [2, 9, 4, 13, 0, 7]
    hq.hq_apply_blocks(st, [(qs, M)], engine="tc_f16")
    oracle.apply_gate(psi, n, qs, M)
    assert rel_l2(st.cpu().numpy().astype(np.complex128), psi) <= 2e-6


def test_sparse_state_zero_groups(hq):
    """|0..0> leaves almost every group all-zero (scale 1 path)."""
    n = 16
    rng = C.SplitMix64(8)
    st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    hq.hq_state_init(st)
    psi = oracle.state_init(n)
    for qs in ([0, 3, 5, 8, 11, 15], [15, 14, 13, 12, 11]):
        M = C.random_unitary(len(qs), rng)
        hq.hq_apply_blocks(st, [(qs, M)], engine="tc_f16")
        oracle.apply_gate(psi, n, qs, M)
    assert rel_l2(st.cpu().numpy().astype(np.complex128), psi) <= 2e-6


@pytest.mark.parametrize("bits", [[0, 1, 2, 3, 4, 5], [6, 7, 8, 9, 10, 11], [1, 3, 4, 8, 10, 12]])
def test_tile_maxima_spanning_many_octaves(hq, bits):
    """Each tile is converted with a provisional power-of-two scale and redone
    when its maximum falls outside the window; tiles whose magnitudes jump by
    up to 2^80 in either direction along a CTA's tile sequence (and by 2^20
    between groups of one tile) must each keep FP32-level error relative to
    their own maximum.  The targets lie in the low 13 flat bits, so every tile
    is one aligned run of 2^13 amplitudes."""
    n, k = 22, 6
    rng = C.SplitMix64(41 + bits[0])
    psi = random_state(n, 17 + bits[0]).reshape(-1, 1 << 13)
    tiles = psi.shape[0]
    tile_exp = np.array([-20 * ((7 * t + (t >> 3)) % 5) for t in range(tiles)])
    within = np.array([-10 * ((i >> 6) % 3) for i in range(1 << 13)])
    psi = (psi * np.exp2(tile_exp)[:, None] * np.exp2(within)[None, :]).reshape(-1)
    st = torch.from_numpy(psi).to(torch.complex64).cuda()
    psi = st.cpu().numpy().astype(np.complex128)  # the oracle starts from the rounded input
    qs = [n - 1 - b for b in bits]
    M = C.random_unitary(k, rng)
    hq.hq_apply_blocks(st, [(qs, M)], engine="tc_f16")
    oracle.apply_gate(psi, n, qs, M)
    got = st.cpu().numpy().astype(np.complex128).reshape(tiles, -1)
    want = psi.reshape(tiles, -1)
    err = np.abs(got - want).max(axis=1) / np.abs(want).max(axis=1)
    assert err.max() <= 2e-6, (int(err.argmax()), float(err.max()))


@pytest.mark.parametrize("method", ["greedy", "dag"])
@pytest.mark.parametrize("kmax", [4, 5, 6])
def test_fused_grid_circuit_fp16_meets_complex64_bar(hq, kmax, method):
    circ = C.random_circuit(C.grid(4, 5), 16, seed=3, two_qubit="fsim")
    want = oracle.simulate(circ)
    blocks = hq.hq_fuse(circ.n, circ.gates, kmax, method=method)
    st = torch.empty(1 << circ.n, dtype=torch.complex64, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, blocks, engine="tc_f16", tc_min_k=4)
    err = rel_l2(st.cpu().numpy().astype(np.complex128), want)
    assert err <= 2e-5 * max(1, len(circ.gates) / 1000), err


def test_fused_grid_circuit_bf16_error_reported(hq):
    circ = C.random_circuit(C.grid(4, 5), 16, seed=3, two_qubit="fsim")
    want = oracle.simulate(circ)
    st = torch.empty(1 << circ.n, dtype=torch.complex64, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, hq.hq_fuse(circ.n, circ.gates, 6), engine="tc_bf16", tc_min_k=4)
    err = rel_l2(st.cpu().numpy().astype(np.complex128), want)
    print(f"bf16 hi+lo relative L2 error over {len(circ.gates)} gates: {err:.3e}")
    assert err <= 5e-3


@pytest.mark.slow
@pytest.mark.parametrize("engine,bar", [("tc_f16", 2e-5), ("cuda_core", 2e-5), ("tc_bf16", 5e-3)])
def test_n28_subset_against_oracle(hq, n28_oracle, engine, bar):
    """Fused k <= 6 blocks (flat bits 0..27 all appear as targets, 24..27
    included) in complex64 against the oracle's complex128 state: FP16 hi+lo
    and the FP32 CUDA-core blocks meet the complex64 bar (relative L2 <= 2e-5
    per 1000 unfused gates); BF16 hi+lo is reported against a loose bound."""
    circ, want = n28_oracle
    G = len(circ.gates)
    st = torch.empty(1 << 28, dtype=torch.complex64, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, hq.hq_fuse(28, circ.gates, 6, method="dag"), engine=engine, tc_min_k=4)
    got = st.cpu().numpy().astype(np.complex128)
    del st
    torch.cuda.empty_cache()
    d = rel_l2(got, want)
    print(f"n=28 subset, {G} gates, {engine} k<=6 vs oracle: rel L2 {d:.3e}")
    assert d <= bar * max(1, G / 1000)


@pytest.mark.slow
def test_n28_subset_per_gate_complex128_against_oracle(hq, n28_oracle):
    """The same circuit gate by gate in complex128 on the GPU: max-abs 1e-12."""
    circ, want = n28_oracle
    st = torch.empty(1 << 28, dtype=torch.complex128, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, circ.gates)
    got = st.cpu().numpy()
    del st
    torch.cuda.empty_cache()
    assert np.abs(got - want).max() <= 1e-12


@pytest.mark.parametrize("bits", [[24, 25, 20, 21, 22, 23], [0, 5, 12, 18, 24, 25], [1, 2, 3, 23, 24, 25]])
def test_targets_on_the_top_flat_bits_n26(hq, bits):
    """One 6-qubit block per case at n = 26 whose targets include flat bits 24
    and 25 (the tile's last box dimensions and the highest run offsets)."""
    n = 26
    rng = C.SplitMix64(301 + bits[2])
    psi = random_state(n, 29 + bits[2])
    st = torch.from_numpy(psi).to(torch.complex64).cuda()
    psi = st.cpu().numpy().astype(np.complex128)
    qs = [n - 1 - b for b in bits]
    M = C.random_unitary(6, rng)
    hq.hq_apply_blocks(st, [(qs, M)], engine="tc_f16")
    oracle.apply_gate(psi, n, qs, M)
    assert rel_l2(st.cpu().numpy().astype(np.complex128), psi) <= 2e-6


@pytest.mark.slow
def test_n33_tc_norm_and_inverse(hq):
    circ = C.config_n33(seed=0)
    G = len(circ.gates)
    blocks = hq.hq_fuse(33, circ.gates, 6)
    st = torch.empty(1 << 33, dtype=torch.complex64, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, blocks, engine="tc_f16")
    nrm = hq.hq_expectation(st, [(1.0, ())]) ** 0.5
    assert abs(nrm - 1) <= 2e-5 * max(1, G / 1000)
    hq.hq_apply_blocks(st, [(q, m.conj().T.copy()) for q, m in reversed(blocks)], engine="tc_f16")
    assert abs(complex(st[0].item()) - 1) <= 4e-5 * max(1, 2 * G / 1000)
    del st
    torch.cuda.empty_cache()
