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
