"""Density matrices on the GPU (Sec. 5 exact noisy simulation; Sec. 2
KrausSuperGate / MatrixSuperGate): rho as the vectorised 2n-qubit state,
every map applied as its superoperator through the state-vector kernels,
against the noise oracle (oracle/noise.py: full 2^n x 2^n matrices) and the
state-vector oracle."""
import functools

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


def random_rho(n, seed):
    rng = np.random.default_rng(seed)  # input only
    A = rng.standard_normal((1 << n, 1 << n)) + 1j * rng.standard_normal((1 << n, 1 << n))
    rho = A @ A.conj().T
    return rho / np.trace(rho)


def oracle_dm(n, ops, tokens=None):
    rho = N.pure_dm(oracle.state_init(n, tokens))
    for kind, qs, m in ops:
        qs = list(qs)
        if kind == "gate":
            rho = N.apply_unitary_dm(rho, n, qs, m)
        elif kind == "kraus":
            rho = N.apply_map(rho, n, qs, m)
        elif kind == "map":
            rho = N.apply_map(rho, n, qs, *m)
        else:
            rho = N.apply_superop(rho, n, qs, m)
    return rho


def noisy_workload(n, depth, seed):
    """Grid circuit with depolarizing and amplitude damping after its gates
    (the noisy-circuit recipe), plus one general map on three qubits and one
    superoperator given directly."""
    circ = C.random_circuit(C.layout_for(n), depth, seed=seed, two_qubit="cz")
    ops = C.noisy_ops(circ, p1=0.02, p2=0.05, gamma=0.03)
    rng = np.random.default_rng(seed)  # input only
    if n >= 3:
        L = [rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8)) for _ in range(2)]
        s = rng.standard_normal((2, 2)) * 0.05
        ops.insert(len(ops) // 2, ("map", (n - 1, 0, 1), (L, None, s)))
    Sd = 0.9 * np.eye(4) + 0.025 * (rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
    ops.append(("super", (n // 2,), Sd))
    return ops


@functools.lru_cache(maxsize=None)
def oracle_case(n):
    ops = noisy_workload(n, 4, seed=n)
    return ops, oracle_dm(n, ops, "+" * n)


def rel_l2(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
@pytest.mark.parametrize("n,tokens", [(1, "+"), (3, None), (5, "+-01+")])
def test_dm_init(hq, dtype, n, tokens):
    rho = torch.empty(1 << n, 1 << n, dtype=getattr(torch, dtype), device="cuda")
    hq.hq_dm_init(rho, tokens)
    want = N.pure_dm(oracle.state_init(n, tokens))
    np.testing.assert_allclose(rho.cpu().numpy(), want, atol=1e-7 if dtype == "complex64" else 1e-15)


CASES = [("complex128", "auto", 0, 1e-12), ("complex128", "auto", 4, 1e-12), ("complex128", "auto", 6, 1e-12),
         ("complex64", "auto", 6, 2e-5), ("complex64", "cuda_core", 6, 2e-5), ("complex64", "tc_f16", 6, 2e-5)]


@pytest.mark.parametrize("dtype,engine,k_max,tol", CASES)
@pytest.mark.parametrize("n", [2, 6, 8])
def test_noisy_circuit_matches_oracle(hq, dtype, engine, k_max, tol, n):
    """Element by element against the oracle's full-matrix evolution; 2n = 16
    vector qubits span several tensor-core and gather tiles.  complex128:
    max-abs 1e-12; complex64: relative L2 2e-5."""
    ops, want = oracle_case(n)
    if 0 < k_max < 6 and any(len(qs) == 3 for _, qs, _ in ops):
        # a 3-qubit map spans 6 vector qubits: refused below k_max = 6
        rho = torch.empty(1 << n, 1 << n, dtype=getattr(torch, dtype), device="cuda")
        with pytest.raises(hq.HQError, match="K_TOO_LARGE"):
            hq.hq_dm_apply(rho, ops, k_max=k_max, engine=engine)
        ops = [o for o in ops if len(o[1]) < 3]
        want = oracle_dm(n, ops, "+" * n)
    rho = torch.empty(1 << n, 1 << n, dtype=getattr(torch, dtype), device="cuda")
    hq.hq_dm_init(rho, "+")
    hq.hq_dm_apply(rho, ops, k_max=k_max, engine=engine)
    got = rho.cpu().numpy().astype(np.complex128)
    if dtype == "complex128":
        assert np.abs(got - want).max() <= tol
    else:
        assert rel_l2(got, want) <= tol


@pytest.mark.parametrize("dtype,tol", [("complex64", 1e-5), ("complex128", 1e-12)])
@pytest.mark.parametrize("n", [1, 5, 9])
def test_dm_expectation_and_purity(hq, dtype, tol, n):
    rho_h = random_rho(n, 100 + n)
    rho = torch.from_numpy(rho_h).to(getattr(torch, dtype)).cuda()
    rho_h = rho.cpu().numpy().astype(np.complex128)
    H = [(1.0, ()), (0.7, ((0, "X"),)), (-0.4, ((n - 1, "Y"),)), (0.3, ((0, "Z"),))]
    if n >= 3:
        H += [(0.25, ((1, "Y"), (2, "Y"))), (-1.5, ((2, "X"), (0, "Y"), (n - 1, "Z"))),
              (0.5, ((1, "Y"), (2, "Y"), (0, "Y")))]
    H += [(0.01 * (t + 1), ((t % n, "XYZ"[t % 3]),)) for t in range(40)]  # more than one launch of terms
    scale = sum(abs(c) for c, _ in H)
    assert abs(hq.hq_dm_expectation(rho, H) - N.dm_expectation(rho_h, H)) <= tol * scale
    assert abs(hq.hq_dm_expectation(rho, [(1.0, ())]) - np.trace(rho_h).real) <= tol
    assert abs(hq.hq_dm_purity(rho) - np.trace(rho_h @ rho_h).real) <= tol


def test_unitary_circuit_gives_pure_state_projector(hq):
    """n = 13 (26 vector qubits): with no noise, rho = |psi><psi| for the
    oracle's state; sampled entries, trace and purity."""
    n = 13
    circ = C.random_circuit(C.layout_for(n), 8, seed=5, two_qubit="fsim")
    psi = oracle.simulate(circ)
    ops = [("gate", g.qubits, g.matrix) for g in circ.gates]
    rho = torch.empty(1 << n, 1 << n, dtype=torch.complex64, device="cuda")
    hq.hq_dm_init(rho)
    hq.hq_dm_apply(rho, ops, k_max=6, engine="tc_f16")
    rng = np.random.default_rng(0)  # input only: the sampled entries
    xs, ys = rng.integers(0, 1 << n, 4096), rng.integers(0, 1 << n, 4096)
    big = np.argsort(-np.abs(psi))[:64]
    xs, ys = np.concatenate([xs, big, big]), np.concatenate([ys, big, np.roll(big, 1)])
    got = rho[torch.from_numpy(xs).cuda(), torch.from_numpy(ys).cuda()].cpu().numpy().astype(np.complex128)
    want = psi[xs] * psi[ys].conj()
    tol = 2e-5 * max(1.0, len(ops) / 1000)
    assert rel_l2(got, want) <= tol
    assert abs(hq.hq_dm_expectation(rho, [(1.0, ())]) - 1) <= tol
    assert abs(hq.hq_dm_purity(rho) - 1) <= 2 * tol
    H = [(1.0, ((0, "Z"),)), (0.5, ((3, "X"), (4, "Y")))]
    assert abs(hq.hq_dm_expectation(rho, H) - oracle.expectation(psi, H)) <= 1e-5 * 1.5


def test_full_size_noisy_dm_properties(hq):
    """The measured workload (n = 15 noisy grid circuit, complex64, fused
    k <= 6 on the tensor cores): unit trace, Hermitian on sampled pairs,
    non-negative diagonal, purity in (1/2^n, 1], and <Z_q> equal to its
    value from the diagonal."""
    n = 15
    circ = C.random_circuit(C.layout_for(n), 10, seed=0, two_qubit="cz")
    ops = C.noisy_ops(circ, p1=1e-3, p2=1e-2, gamma=1e-3)
    rho = torch.empty(1 << n, 1 << n, dtype=torch.complex64, device="cuda")
    hq.hq_dm_init(rho)
    hq.hq_dm_apply(rho, ops, k_max=6, engine="tc_f16")
    tr = hq.hq_dm_expectation(rho, [(1.0, ())])
    assert abs(tr - 1) <= 2e-5
    rng = np.random.default_rng(1)  # input only
    xs = torch.from_numpy(rng.integers(0, 1 << n, 4096)).cuda()
    ys = torch.from_numpy(rng.integers(0, 1 << n, 4096)).cuda()
    a, b = rho[xs, ys], rho[ys, xs].conj()
    assert float((a - b).abs().max()) <= 2e-5 * float(rho.diagonal().abs().max())
    diag = rho.diagonal().real.double()
    assert float(diag.min()) >= -1e-6
    pur = hq.hq_dm_purity(rho)
    assert 1.0 / (1 << n) < pur <= 1 + 1e-5
    idx = torch.arange(1 << n, device="cuda")
    for q in (0, 7, n - 1):
        sign = 1 - 2 * ((idx >> (n - 1 - q)) & 1).double()
        zq = float((diag * sign).sum())
        assert abs(hq.hq_dm_expectation(rho, [(1.0, ((q, "Z"),))]) - zq) <= 1e-6


def test_many_unfusable_maps(hq):
    """125 two-qubit maps along a chain, none of which can share a 4-vector-
    qubit block with its neighbours: more blocks than the first fusion
    attempt makes room for, so the library fuses again with room for all;
    complex128 against the oracle."""
    n = 6
    srng = C.SplitMix64(31)
    ops = []
    for r in range(25):
        for i in range(n - 1):
            U = C.random_unitary(2, srng)
            ops.append(("gate", (i, i + 1), U) if r % 2 else ("kraus", (i, i + 1), [np.sqrt(0.9) * U,
                                                                                     np.sqrt(0.1) * np.eye(4)]))
    want = oracle_dm(n, ops, "+" * n)
    rho = torch.empty(1 << n, 1 << n, dtype=torch.complex128, device="cuda")
    hq.hq_dm_init(rho, "+")
    hq.hq_dm_apply(rho, ops, k_max=4)
    assert np.abs(rho.cpu().numpy() - want).max() <= 1e-12
    blocks = hq.hq_fuse(2 * n, [(tuple(qs) + tuple(n + q for q in qs), hq.hq_dm_superop([m] if k == "gate" else m))
                                for k, qs, m in ops], 4, method="dag", restarts=8, seed=0)
    assert len(blocks) > 64 + len(ops) // 4
