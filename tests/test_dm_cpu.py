"""Host-side checks of the density-matrix entry points: the superoperator
builder (hq_dm_superop) against the vectorisation identity and the noise
oracle, and argument validation before any device work."""
import ctypes

import numpy as np
import pytest

from oracle import noise as N
from paper_2111_06868_gb300 import circuits as C


@pytest.fixture(scope="module")
def hq():
    from paper_2111_06868_gb300 import build
    from paper_2111_06868_gb300 import hq as _hq

    build.build()
    _hq.load()
    return _hq


def _ops(k, count, rng):
    d = 1 << k
    return [rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d)) for _ in range(count)]


@pytest.mark.parametrize("k", [1, 2, 3])
def test_superop_is_the_vectorised_map(hq, k):
    """S applied to vec(rho) gives the oracle's sum_ij s_ij L_i rho R_j^dag
    (full matrices), for random non-Hermitian operators and coefficients."""
    rng = np.random.default_rng(k)  # input only
    L, R = _ops(k, 3, rng), _ops(k, 2, rng)
    s = rng.standard_normal((3, 2)) + 1j * rng.standard_normal((3, 2))
    S = hq.hq_dm_superop(L, R, s)
    d = 1 << k
    A = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    want = N.apply_map(A, k, list(range(k)), L, R, s)
    np.testing.assert_allclose((S @ A.reshape(-1)).reshape(d, d), want, atol=1e-12)


def test_superop_defaults_kraus_and_gate(hq):
    rng = C.SplitMix64(4)
    U = C.random_unitary(2, rng)
    np.testing.assert_allclose(hq.hq_dm_superop([U]), np.kron(U, U.conj()), atol=0)
    ks = C.depolarizing(0.3, 1)
    S = hq.hq_dm_superop(ks)
    # trace preservation: vec(I)^T S = vec(I)^T
    vI = np.eye(2).reshape(-1)
    np.testing.assert_allclose(vI @ S, vI, atol=1e-15)
    # full depolarization maps everything to Tr(rho) I / 2
    np.testing.assert_allclose(hq.hq_dm_superop(C.depolarizing(1.0, 1)), np.outer(vI, vI) / 2, atol=1e-15)


def test_dm_validation_before_any_device_work(hq):
    lib = hq.load()
    fake = ctypes.c_void_p(1 << 20)
    out = ctypes.c_double()
    assert lib.hq_dm_init(None, 3, 0, None, None) == -1
    assert lib.hq_dm_init(fake, 18, 0, None, None) == -5          # 2n > 34
    assert lib.hq_dm_init(fake, 0, 0, None, None) == -5
    assert lib.hq_dm_init(fake, 3, 0, b"0x1", None) == -10
    assert lib.hq_dm_init(ctypes.c_void_p((1 << 20) + 8), 3, 0, None, None) == -13
    assert lib.hq_dm_purity(fake, 3, 5, ctypes.byref(out), None) == -6
    U = np.eye(2, dtype=np.complex128)
    op = hq.hq_dm_op()
    op.kind, op.k, op.nl, op.left = hq.HQ_DM_MAP, 1, 1, U.ctypes.data
    op.qubits[0] = 3
    assert lib.hq_dm_apply(fake, 3, 0, ctypes.byref(op), 1, 6, None, None) == -2   # qubit range
    op.qubits[0] = 0
    op.k = 4
    assert lib.hq_dm_apply(fake, 5, 0, ctypes.byref(op), 1, 6, None, None) == -4   # k > 3
    op.k = 1
    assert lib.hq_dm_apply(fake, 3, 0, ctypes.byref(op), 1, 7, None, None) == -12  # k_max
    assert lib.hq_dm_apply(fake, 3, 0, ctypes.byref(op), -1, 6, None, None) == -12
    op.kind = 9
    assert lib.hq_dm_apply(fake, 3, 0, ctypes.byref(op), 1, 6, None, None) == -12
    op.kind, op.nl = hq.HQ_DM_MAP, 0
    assert lib.hq_dm_apply(fake, 3, 0, ctypes.byref(op), 1, 6, None, None) == -12
    op.nl, op.nr, op.right = 1, 2, U.ctypes.data  # s NULL needs nl == nr
    assert lib.hq_dm_apply(fake, 3, 0, ctypes.byref(op), 1, 6, None, None) == -12
    op.nr, op.right = 0, None
    op2 = (hq.hq_dm_op * 1)()
    op2[0] = op
    op2[0].k, op2[0].qubits[1] = 2, 1
    U4 = np.eye(4, dtype=np.complex128)
    op2[0].left = U4.ctypes.data
    assert lib.hq_dm_apply(fake, 3, 0, op2, 1, 3, None, None) == -4  # 2k = 4 > k_max = 3
    S = np.zeros(2, np.float64)
    assert lib.hq_dm_superop(1, 1, None, 0, None, None, S.ctypes.data_as(ctypes.c_void_p)) == -1
    assert lib.hq_dm_superop(4, 1, U.ctypes.data_as(ctypes.c_void_p), 0, None, None,
                             S.ctypes.data_as(ctypes.c_void_p)) == -4


@pytest.mark.parametrize("name,ks", [("depolarizing1", C.depolarizing(0.3, 1)), ("depolarizing2", C.depolarizing(0.2, 2)),
                                     ("dephasingX", C.dephasing(0.4, "X")), ("dephasingY", C.dephasing(0.1, "Y")),
                                     ("amplitude_damping", C.amplitude_damping(0.3)),
                                     ("generalized_damping", C.amplitude_damping(0.2, 0.15))])
def test_channel_superops_preserve_trace(hq, name, ks):
    """Every channel of Sec. 2.1 is trace preserving: vec(I)^T S = vec(I)^T;
    Pauli channels are also unital: S vec(I) = vec(I); and the channel with
    operators {K^dag} is the Hilbert-Schmidt adjoint of the one with {K}:
    Tr(A^dag Lambda(B)) = Tr(Lambda*(A)^dag B)."""
    S = hq.hq_dm_superop(ks)
    d = ks[0].shape[0]
    vI = np.eye(d).reshape(-1)
    np.testing.assert_allclose(vI @ S, vI, atol=1e-14)
    if not name.endswith("damping"):
        np.testing.assert_allclose(S @ vI, vI, atol=1e-14)
    Sa = hq.hq_dm_superop([K.conj().T for K in ks])
    # Tr(A^dag Lambda(B)) = Tr(Lambda*(A)^dag B) for random A, B
    rng = np.random.default_rng(d)  # input only
    A = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    B = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    lhs = np.vdot(A.reshape(-1), S @ B.reshape(-1))
    rhs = np.vdot(Sa @ A.reshape(-1), B.reshape(-1))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_fused_superops_reproduce_the_oracle_density_matrix(hq):
    """A noisy circuit at the density-matrix level on the host: every gate
    and channel as its superoperator on vector qubits (q, n + q), fused by
    hq_fuse_dag into <= 6-qubit blocks, applied to vec(rho) by the
    state-vector oracle, equals the noise oracle's full-matrix evolution."""
    import oracle

    n = 4
    circ = C.random_circuit(C.layout_for(n), 4, seed=3, two_qubit="cz")
    ops = C.noisy_ops(circ, p1=0.05, p2=0.1, gamma=0.07)
    rho = N.pure_dm(oracle.state_init(n, "+0-1"))
    for kind, qs, m in ops:
        rho = N.apply_unitary_dm(rho, n, list(qs), m) if kind == "gate" else N.apply_map(rho, n, list(qs), m)
    sup = [(tuple(qs) + tuple(n + q for q in qs), hq.hq_dm_superop([m] if kind == "gate" else m))
           for kind, qs, m in ops]
    blocks = hq.hq_fuse(2 * n, sup, 6, method="dag", restarts=8, seed=0)
    assert len(blocks) < len(sup)
    v = N.pure_dm(oracle.state_init(n, "+0-1")).reshape(-1).copy()
    for qs, M in blocks:
        v = oracle.apply_gate(v, 2 * n, qs, M)
    np.testing.assert_allclose(v.reshape(1 << n, 1 << n), rho, atol=1e-13)
