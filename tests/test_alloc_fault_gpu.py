"""Error paths on the GPU without a GPU fault: a scratch allocation that
fails (injected through hq_test_fail_next_allocs, as if the device were out
of memory) makes the entry point return HQ_ERR_ALLOC, leaves the state as it
was, and the next call succeeds with the right answer."""
import numpy as np
import pytest

import oracle
from oracle import noise as N
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
    yield _hq
    _hq.hq_test_fail_next_allocs(0)


def expect_alloc_error(hq, call):
    hq.hq_test_fail_next_allocs(1)
    try:
        with pytest.raises(hq.HQError) as e:
            call()
        assert e.value.name == "HQ_ERR_ALLOC"
    finally:
        hq.hq_test_fail_next_allocs(0)


def test_injection_argument_check(hq):
    with pytest.raises(hq.HQError, match="HQ_ERR_ARG"):
        hq.hq_test_fail_next_allocs(-1)


@pytest.mark.parametrize("dtype,tol", [("complex64", 1e-5), ("complex128", 1e-12)])
def test_expectation_and_noise_paths_report_and_recover(hq, dtype, tol):
    n = 14
    rng = np.random.default_rng(5)  # input only
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    st = torch.from_numpy(psi).to(getattr(torch, dtype)).cuda()
    psi = st.cpu().numpy().astype(np.complex128)
    # one X-mask group (streaming kernel) and several (tiled kernel)
    for H in ([(1.0, ((3, "X"),))], C.ansatz_hamiltonian(n)):
        expect_alloc_error(hq, lambda: hq.hq_expectation(st, H))
        scale = sum(abs(c) for c, _ in H)
        assert abs(hq.hq_expectation(st, H) - oracle.expectation(psi, H)) <= tol * scale
    # reduced density matrix
    expect_alloc_error(hq, lambda: hq.hq_reduced_density_matrix(st, (2,)))
    rho2 = hq.hq_reduced_density_matrix(st, (2,))
    assert abs(np.trace(rho2).real - 1) <= 10 * tol
    # a state-dependent channel: nothing applied when its scratch fails
    before = st.clone()
    ops = [("kraus", (1,), C.amplitude_damping(0.3))]
    expect_alloc_error(hq, lambda: hq.hq_run_trajectory(st, ops, np.array([0.5])))
    torch.cuda.synchronize()
    assert torch.equal(st, before)
    i, want = N.trajectory_step(psi, n, [1], C.amplitude_damping(0.3), 0.5)
    got = hq.hq_run_trajectory(st, ops, np.array([0.5]))
    assert got.tolist() == [i]
    assert np.abs(st.cpu().numpy().astype(np.complex128) - want).max() <= 2 * tol


def test_density_matrix_expectation_reports_and_recovers(hq):
    n = 3
    rho = torch.empty(1 << n, 1 << n, dtype=torch.complex128, device="cuda")
    hq.hq_dm_init(rho, "+")
    H = [(1.0, ((0, "X"),)), (0.5, ((1, "Z"),))]
    expect_alloc_error(hq, lambda: hq.hq_dm_expectation(rho, H))
    assert abs(hq.hq_dm_expectation(rho, H) - 1.0) <= 1e-12


def seeded_state(n, seed, dtype):
    rng = np.random.default_rng(seed)  # input only
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    st = torch.from_numpy(psi).to(getattr(torch, dtype)).cuda()
    return st, st.cpu().numpy().astype(np.complex128)


def rel_l2(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


@pytest.mark.parametrize("engine", ["tc_f16", "tc_pass"])
def test_tensor_core_matrix_buffer_reports_and_leaves_state(hq, engine):
    """The tensor-core and tile-pass engines take their matrix buffer before
    enqueueing any kernel: HQ_ERR_ALLOC leaves the state untouched."""
    n = 15
    st, psi = seeded_state(n, 7, "complex64")
    rng = C.SplitMix64(3)
    blocks = [((0, 3, 5, 8, 11, 14), C.random_unitary(6, rng)), ((1, 2, 4, 9, 12, 13), C.random_unitary(6, rng))]
    before = st.clone()
    expect_alloc_error(hq, lambda: hq.hq_apply_blocks(st, blocks, engine=engine))
    torch.cuda.synchronize()
    assert torch.equal(st, before)
    hq.hq_apply_blocks(st, blocks, engine=engine)
    for qs, m in blocks:
        oracle.apply_gate(psi, n, qs, m)
    assert rel_l2(st.cpu().numpy().astype(np.complex128), psi) <= 2e-6


@pytest.mark.parametrize("dtype,tol", [("complex64", 2e-6), ("complex128", 1e-12)])
def test_cuda_core_block_list_applies_the_prefix(hq, dtype, tol):
    """CUDA-core wide blocks allocate one matrix copy each: after HQ_ERR_ALLOC
    the blocks before the failing one have been applied and none after."""
    n = 13
    st, psi = seeded_state(n, 11, dtype)
    rng = C.SplitMix64(5)
    blocks = [((2, 7), C.random_unitary(2, rng)), ((0, 1, 4, 6, 9), C.random_unitary(5, rng)),
              ((3, 5, 8, 10, 11, 12), C.random_unitary(6, rng))]
    expect_alloc_error(hq, lambda: hq.hq_apply_blocks(st, blocks, engine="cuda_core"))
    oracle.apply_gate(psi, n, *blocks[0])
    got = st.cpu().numpy().astype(np.complex128)
    err = np.abs(got - psi).max() if dtype == "complex128" else rel_l2(got, psi)
    assert err <= tol
    hq.hq_apply_blocks(st, blocks[1:], engine="cuda_core")
    for qs, m in blocks[1:]:
        oracle.apply_gate(psi, n, qs, m)
    got = st.cpu().numpy().astype(np.complex128)
    err = np.abs(got - psi).max() if dtype == "complex128" else rel_l2(got, psi)
    assert err <= tol


def test_kraus_sampled_reports_and_recovers(hq):
    """A state-dependent channel whose scratch fails is not applied; the next
    call samples the oracle's branch."""
    n = 12
    st, psi = seeded_state(n, 13, "complex128")
    K = C.amplitude_damping(0.4)
    before = st.clone()
    expect_alloc_error(hq, lambda: hq.hq_apply_kraus_sampled(st, (4,), K, 0.3))
    torch.cuda.synchronize()
    assert torch.equal(st, before)
    i, want = N.trajectory_step(psi, n, [4], K, 0.3)
    assert hq.hq_apply_kraus_sampled(st, (4,), K, 0.3) == i
    assert np.abs(st.cpu().numpy() - want).max() <= 1e-12
