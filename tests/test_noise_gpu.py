"""Noisy paths on the GPU (Sec. 5): reduced density matrices, pure-state
sampling of Kraus channels and whole trajectories, against the noise oracle
(oracle/noise.py) and the state-vector oracle."""
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
    return _hq


def random_state(n, seed):
    rng = np.random.default_rng(seed)  # input only
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return psi / np.linalg.norm(psi)


def rdm_of(psi, n, qubits):
    """Reduced density matrix by reshaping (qubits first, in the given order)."""
    t = psi.reshape((2,) * n)
    rest = [q for q in range(n) if q not in qubits]
    t = np.moveaxis(t, list(qubits) + rest, list(range(n))).reshape(1 << len(qubits), -1)
    return t @ t.conj().T


@pytest.mark.parametrize("dtype,tol", [("complex64", 2e-6), ("complex128", 1e-13)])
@pytest.mark.parametrize("n", [12, 19])
def test_reduced_density_matrix(hq, dtype, tol, n):
    psi = random_state(n, n)
    st = torch.from_numpy(psi).to(getattr(torch, dtype)).cuda()
    psi = st.cpu().numpy().astype(np.complex128)
    for qs in [(0,), (n - 1,), (n - 2, 3), (n - 1, n - 2), (5, 1)]:
        got = hq.hq_reduced_density_matrix(st, qs)
        np.testing.assert_allclose(got, rdm_of(psi, n, list(qs)), atol=tol)


CHANNELS = [("ad", lambda: N.amplitude_damping_kraus(0.3)), ("gad", lambda: N.amplitude_damping_kraus(0.2, 0.1)),
            ("dep1", lambda: N.depolarizing_kraus(0.4)), ("deph", lambda: N.dephasing_kraus(0.3, "X")),
            ("dep2", lambda: N.depolarizing_kraus(0.5, 2))]


@pytest.mark.parametrize("name,make", CHANNELS)
def test_kraus_sampling_step_matches_oracle(hq, name, make):
    """complex128: with the same uniforms the GPU picks the oracle's branch
    and leaves the oracle's state."""
    n = 11
    ks = make()
    k = int(ks[0].shape[0]).bit_length() - 1
    rng = np.random.default_rng(3)  # input only: the uniforms
    psi = random_state(n, 7)
    st = torch.from_numpy(psi).cuda()
    for step in range(12):
        qs = [(step * 5) % n, (step * 3 + 1) % n][:k] if k == 2 else [(step * 5) % n]
        if k == 2 and qs[0] == qs[1]:
            qs[1] = (qs[1] + 1) % n
        u = float(rng.random())
        i_want, psi = N.trajectory_step(psi, n, qs, ks, u)
        i_got = hq.hq_apply_kraus_sampled(st, qs, ks, u)
        assert i_got == i_want, (step, u)
    assert np.abs(st.cpu().numpy() - psi).max() <= 1e-12


def noisy_circuit(n, depth, seed):
    circ = C.random_circuit(C.layout_for(n), depth, seed=seed, two_qubit="cz")
    return C.noisy_ops(circ, p1=0.02, p2=0.05, gamma=0.03)


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
def test_trajectory_matches_oracle_trajectory(hq, dtype):
    n = 10
    ops = noisy_circuit(n, 6, 1)
    nch = sum(1 for o in ops if o[0] == "kraus")
    u = np.random.default_rng(2).random(nch)  # input only
    psi = oracle.state_init(n)
    want, c = [], 0
    for kind, qs, m in ops:
        if kind == "gate":
            psi = oracle.apply_gate(psi, n, qs, m)
        else:
            i, psi = N.trajectory_step(psi, n, list(qs), m, u[c])
            want.append(i)
            c += 1
    st = torch.zeros(1 << n, dtype=getattr(torch, dtype), device="cuda")
    hq.hq_state_init(st)
    got = hq.hq_run_trajectory(st, ops, u)
    assert got.tolist() == want
    err = np.abs(st.cpu().numpy().astype(np.complex128) - psi).max()
    assert err <= (1e-12 if dtype == "complex128" else 2e-6)


def test_trajectory_average_converges_to_density_matrix(hq):
    """<Z_0> and <X_2> averaged over GPU trajectories agree with the exact
    density-matrix evolution within five standard errors."""
    n = 5
    ops = noisy_circuit(n, 5, 4)
    rho = N.pure_dm(oracle.state_init(n))
    for kind, qs, m in ops:
        rho = N.apply_unitary_dm(rho, n, list(qs), m) if kind == "gate" else N.apply_map(rho, n, list(qs), m)
    H = [(1.0, ((0, "Z"),)), (0.5, ((2, "X"),))]
    exact = N.dm_expectation(rho, H)
    nch = sum(1 for o in ops if o[0] == "kraus")
    rng = np.random.default_rng(9)  # input only
    st = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    vals = []
    for _ in range(600):
        hq.hq_state_init(st)
        hq.hq_run_trajectory(st, ops, rng.random(nch))
        vals.append(hq.hq_expectation(st, H))
    vals = np.array(vals)
    assert abs(vals.mean() - exact) <= 5 * vals.std() / np.sqrt(len(vals)) + 1e-12


def random_kraus(k, nK, rng):
    """nK Kraus operators on k qubits from a random isometry (sum K^dag K = I)."""
    D = 1 << k
    A = rng.standard_normal((nK * D, D)) + 1j * rng.standard_normal((nK * D, D))
    Q, _ = np.linalg.qr(A)
    return [Q[i * D:(i + 1) * D, :] for i in range(nK)]


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
def test_trajectory_folds_gates_into_two_qubit_channels(hq, dtype):
    """State-dependent two-qubit channels right after gates on the same
    qubits (which the library folds into the channel's sampling) and after
    gates on the same qubits in the other order or on other qubits (which it
    applies on their own): branches and states against the oracle."""
    n = 9
    rng = np.random.default_rng(21)  # input only
    srng = C.SplitMix64(5)
    U = [C.random_unitary(2, srng) for _ in range(4)]
    V = C.random_unitary(1, srng)
    ops = [("gate", (2, 5), U[0]), ("gate", (2, 5), U[1]), ("kraus", (2, 5), random_kraus(2, 3, rng)),
           ("gate", (5, 2), U[2]), ("kraus", (2, 5), random_kraus(2, 2, rng)),
           ("gate", (7, 0), U[3]), ("gate", (3,), V), ("kraus", (0, 7), random_kraus(2, 4, rng)),
           ("gate", (3,), V), ("kraus", (3,), C.depolarizing(0.3, 1)), ("kraus", (3,), random_kraus(1, 3, rng)),
           ("kraus", (2, 5), random_kraus(2, 2, rng))]
    psi0 = oracle.state_init(n, "+-01+-01+")
    for trial in range(4):
        u = rng.random(sum(1 for o in ops if o[0] == "kraus"))
        psi, want, c = psi0.copy(), [], 0
        for kind, qs, m in ops:
            if kind == "gate":
                psi = oracle.apply_gate(psi, n, qs, m)
            else:
                i, psi = N.trajectory_step(psi, n, list(qs), m, u[c])
                want.append(i)
                c += 1
        st = torch.empty(1 << n, dtype=getattr(torch, dtype), device="cuda")
        hq.hq_state_init(st, "+-01+-01+")
        got = hq.hq_run_trajectory(st, ops, u)
        assert got.tolist() == want, trial
        err = np.abs(st.cpu().numpy().astype(np.complex128) - psi).max()
        assert err <= (1e-12 if dtype == "complex128" else 2e-6), (trial, err)
