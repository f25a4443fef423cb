"""GPU parity: libhq.so (through the C ABI) against the CPU oracle on the same
seeded inputs.  Tolerances: complex128 max-abs <= 1e-12; complex64 relative L2
<= 2e-5 * max(1, G/1000) with G the number of unfused gates."""
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


DT = {"c64": torch.complex64, "c128": torch.complex128}


def to_dev(psi, dt):
    return torch.from_numpy(psi.astype(np.complex128)).to(DT[dt]).cuda()


def to_host(t):
    return t.cpu().numpy().astype(np.complex128)


def assert_close(got, want, dt, G=1):
    if dt == "c128":
        err = np.max(np.abs(got - want))
        assert err <= 1e-12, f"max-abs {err:.3e}"
    else:
        rel = np.linalg.norm(got - want) / np.linalg.norm(want)
        tol = 2e-5 * max(1.0, G / 1000)
        assert rel <= tol, f"rel L2 {rel:.3e} > {tol:.1e}"


def random_state(n, seed):
    """Seeded normalised Gaussian state (input only)."""
    rng = C.SplitMix64(seed)
    v = np.empty(2 << n)
    for i in range(0, v.size, 2):
        u1, u2 = max(rng.uniform(), 1e-300), rng.uniform()
        r = math.sqrt(-2 * math.log(u1))
        v[i], v[i + 1] = r * math.cos(2 * math.pi * u2), r * math.sin(2 * math.pi * u2)
    psi = v[0::2] + 1j * v[1::2]
    return psi / np.linalg.norm(psi)


# --------------------------------------------------------------------------
@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("tokens", ["0", "1", "+", "-", "01+-", "+-+-10+"])
@pytest.mark.parametrize("n", [1, 3, 7, 13])
def test_state_init(hq, dt, tokens, n):
    tok = (tokens * n)[:n]
    st = torch.empty(1 << n, dtype=DT[dt], device="cuda")
    hq.hq_state_init(st, tok)
    assert_close(to_host(st), oracle.state_init(n, tok), dt)


def qubit_sets(n, k, seed):
    rng = C.SplitMix64(seed)
    sets = [list(range(n - k, n)),             # lowest bits (qubits n-1..)
            list(range(k)),                    # highest bits
            list(range(n - 1, n - 1 - k, -1))]  # lowest bits, reversed order
    rnd = []
    while len(rnd) < k:
        q = rng.randint(0, n - 1)
        if q not in rnd:
            rnd.append(q)
    sets.append(rnd)
    if k >= 2:
        sets.append([n - 1] + list(range(k - 1)))  # mixed: one low bit, the rest high
    return sets


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("n", [6, 9, 13, 17])
def test_apply_gate_every_position_class(hq, dt, k, n):
    if k > n:
        pytest.skip()
    rng = C.SplitMix64(1000 * n + k)
    psi = random_state(n, n * 31 + k)
    st = to_dev(psi, dt)
    want = psi.copy()
    for qs in qubit_sets(n, k, n + 7 * k):
        M = C.random_unitary(k, rng)
        hq.hq_apply_gate(st, qs, M)
        oracle.apply_gate(want, n, qs, M)
    assert_close(to_host(st), want, dt, G=5)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_apply_gate_many_tiles_per_cta(hq, dt, k):
    """n = 22: 1024 (complex64) or 2048 (complex128) tiles, more than the
    CTAs of one launch, so every CTA takes several tiles (and the complex64
    gather kernel's copy of the next tile overlaps the current one)."""
    n = 22
    rng = C.SplitMix64(4200 + k)
    g = np.random.default_rng(77 + k)  # input only
    psi = g.standard_normal(1 << n) + 1j * g.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    st = to_dev(psi, dt)
    sets = qubit_sets(n, k, 5 * k)
    for qs in sets:
        M = C.random_unitary(k, rng)
        # and a monomial gate (permutation times phases: the permute-and-phase kernel)
        P = np.zeros((1 << k, 1 << k), np.complex128)
        P[np.arange(1 << k), g.permutation(1 << k)] = np.exp(2j * np.pi * g.random(1 << k))
        for A in (M, P):
            hq.hq_apply_gate(st, qs, A)
            oracle.apply_gate(psi, n, qs, A)
    assert_close(to_host(st), psi, dt, G=2 * len(sets))


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("k", [1, 2, 3, 6])
def test_apply_gate_k_equals_n(hq, dt, k):
    n = k
    rng = C.SplitMix64(77 + k)
    psi = random_state(n, 5 + k)
    M = C.random_unitary(k, rng)
    qs = list(range(n))[::-1]
    st = to_dev(psi, dt)
    hq.hq_apply_gate(st, qs, M)
    oracle.apply_gate(psi, n, qs, M)
    assert_close(to_host(st), psi, dt)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_diagonal_gates(hq, dt, k):
    n = 14
    rng = C.SplitMix64(500 + k)
    psi = random_state(n, 900 + k)
    st = to_dev(psi, dt)
    for qs in qubit_sets(n, k, 3 * k):
        d = np.exp(2j * math.pi * np.array([rng.uniform() for _ in range(1 << k)]))
        M = np.diag(d)
        hq.hq_apply_gate(st, qs, M)
        oracle.apply_gate(psi, n, qs, M)
    assert_close(to_host(st), psi, dt, G=5)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("kmax", [0, 2, 3, 4, 5, 6])
def test_circuit_n12_per_gate_and_fused(hq, dt, kmax):
    circ = C.config_small(seed=1)
    want = oracle.simulate(circ)
    st = torch.empty(1 << circ.n, dtype=DT[dt], device="cuda")
    hq.hq_state_init(st)
    blocks = hq.hq_fuse(circ.n, circ.gates, kmax) if kmax else circ.gates
    hq.hq_apply_blocks(st, blocks)
    assert_close(to_host(st), want, dt, G=len(circ.gates))


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("kmax", [0, 4])
def test_circuit_grid_fsim_n20(hq, dt, kmax):
    """4x5 grid, depth 12, fSim entanglers: spans many tiles and every bit class."""
    circ = C.random_circuit(C.grid(4, 5), 12, seed=11, two_qubit="fsim")
    want = oracle.simulate(circ, tokens="+")
    st = torch.empty(1 << circ.n, dtype=DT[dt], device="cuda")
    hq.hq_state_init(st, "+")
    blocks = hq.hq_fuse(circ.n, circ.gates, kmax) if kmax else circ.gates
    hq.hq_apply_blocks(st, blocks)
    assert_close(to_host(st), want, dt, G=len(circ.gates))


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_dense_circuit_wide_blocks(hq, dt):
    """Random dense gates fused up to 6 qubits (CUDA-core block kernel)."""
    circ = C.random_dense_circuit(15, 60, seed=4, kmax=3)
    psi0 = random_state(15, 12)
    want = oracle.apply_circuit(psi0.copy(), circ)
    st = to_dev(psi0, dt)
    hq.hq_apply_blocks(st, hq.hq_fuse(15, circ.gates, 6), engine="cuda_core")
    assert_close(to_host(st), want, dt, G=60)


def test_empty_block_list_is_identity(hq):
    psi = random_state(10, 3)
    st = to_dev(psi, "c128")
    hq.hq_apply_blocks(st, [])
    assert_close(to_host(st), psi, "c128")


# --------------------------------------------------------------------------
# expectation
# --------------------------------------------------------------------------
def random_hamiltonian(n, T, seed):
    rng = C.SplitMix64(seed)
    H = []
    for _ in range(T):
        L = rng.randint(0, min(4, n))
        qs = []
        while len(qs) < L:
            q = rng.randint(0, n - 1)
            if q not in qs:
                qs.append(q)
        H.append((rng.uniform() - 0.5, tuple((q, "XYZ"[rng.randint(0, 2)]) for q in qs)))
    return H


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 2, 5, 11, 16])
def test_expectation_random_pauli_sums(hq, dt, n):
    psi = random_state(n, 40 + n)
    H = random_hamiltonian(n, 12, 7 * n)
    want = oracle.expectation(psi, H)
    got = hq.hq_expectation(to_dev(psi, dt), H)
    tol = 1e-12 if dt == "c128" else 1e-5 * max(1.0, sum(abs(c) for c, _ in H))
    assert abs(got - want) <= tol


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_expectation_norm_and_ansatz_hamiltonian(hq, dt):
    n = 14
    circ = C.ansatz(n, 2)
    th = C.ansatz_params(circ.n_params, 1, 3)[0]
    psi = oracle.simulate(circ, theta=th)
    st = to_dev(psi, dt)
    H = C.ansatz_hamiltonian(n)
    tol = 1e-12 if dt == "c128" else 2e-5
    assert abs(hq.hq_expectation(st, [(1.0, ())]) - 1.0) <= tol
    assert abs(hq.hq_expectation(st, H) - oracle.expectation(psi, H)) <= tol * 10


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n,seed", [(13, 1), (17, 2), (20, 3)])
def test_expectation_tiled_passes(hq, dt, n, seed):
    """Pauli sums whose X masks reach the high qubits: one read of the state per
    tile pass (low tile, then 7 low bits + up to 6 high bits), signs from the
    tile base folded per tile."""
    rng = C.SplitMix64(seed)
    psi = random_state(n, 60 + n)
    H = [(0.5, ((q, "Z"), ((q + 1) % n, "Z"))) for q in range(n)]
    H += [(rng.uniform() - 0.5, ((q, "X"),)) for q in range(n)]
    H += [(rng.uniform() - 0.5, ((q, "Y"), ((q + 5) % n, "X"), ((q + 9) % n, "Z"))) for q in range(0, n, 3)]
    H += [(0.25, ())]
    want = oracle.expectation(psi, H)
    got = hq.hq_expectation(to_dev(psi, dt), H)
    tol = 1e-12 if dt == "c128" else 1e-5 * max(1.0, sum(abs(c) for c, _ in H))
    assert abs(got - want) <= tol


def test_expectation_term_wider_than_a_tile_pass(hq):
    """A term whose X mask needs more high bits than a tile pass holds sends
    the sum to the per-group kernel."""
    n = 18
    psi = random_state(n, 71)
    H = [(0.3, tuple((q, "X") for q in range(8))), (0.2, ((17, "Z"),)), (0.1, ((0, "X"),))]
    for dt in ("c64", "c128"):
        got = hq.hq_expectation(to_dev(psi, dt), H)
        tol = 1e-12 if dt == "c128" else 1e-5
        assert abs(got - oracle.expectation(psi, H)) <= tol


def test_expectation_many_groups(hq):
    """More xmask groups and terms than one parameter block holds."""
    n = 12
    psi = random_state(n, 99)
    H = [(0.1 * (i + 1), ((i % n, "X"), ((i + 3) % n, "Y"))) for i in range(40)]
    H += [(0.05, ((q, "Z"),)) for q in range(n)] * 9
    assert abs(hq.hq_expectation(to_dev(psi, "c128"), H) - oracle.expectation(psi, H)) <= 1e-12


# --------------------------------------------------------------------------
# errors come back as status codes, before any work is enqueued
# --------------------------------------------------------------------------
def test_argument_errors(hq):
    st = torch.zeros(1 << 5, dtype=torch.complex64, device="cuda")
    M = np.eye(2)
    with pytest.raises(hq.HQError, match="QUBIT_RANGE"):
        hq.hq_apply_gate(st, [5], M)
    with pytest.raises(hq.HQError, match="DUP_QUBIT"):
        hq.hq_apply_gate(st, [1, 1], np.eye(4))
    with pytest.raises(hq.HQError, match="K_TOO_LARGE"):
        hq.hq_apply_gate(st, list(range(5)) + [0], np.eye(64))
    with pytest.raises(hq.HQError, match="TOKEN"):
        hq.hq_state_init(st, "0+x01")
    m = np.eye(2, dtype=np.complex128)
    q = (hq.ctypes.c_int * 1)(0)
    rc = hq.load().hq_apply_gate(hq.ctypes.c_void_p(st.data_ptr() + 8), 5, hq.HQ_C64, q, 1,
                                 m.ctypes.data_as(hq.ctypes.c_void_p), None)
    assert hq.STATUS[rc] == "HQ_ERR_ALIGN"


# --------------------------------------------------------------------------
# full-size properties (n = 30): norm, and C followed by C^+ returns |0..0>
# --------------------------------------------------------------------------
@pytest.mark.slow
def test_n30_fused_norm_and_inverse(hq):
    circ = C.config_n30(seed=0)
    G = len(circ.gates)
    blocks = hq.hq_fuse(circ.n, circ.gates, 4)
    st = torch.empty(1 << 30, dtype=torch.complex64, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, blocks)
    assert abs(hq.hq_expectation(st, [(1.0, ())]) ** 0.5 - 1.0) <= 2e-5 * max(1, G / 1000)
    inv = [(q, m.conj().T.copy()) for q, m in reversed(blocks)]
    hq.hq_apply_blocks(st, inv)
    a0 = complex(st[0].item())
    assert abs(a0 - 1.0) <= 2 * 2e-5 * max(1, 2 * G / 1000)
    del st
    torch.cuda.empty_cache()


@pytest.mark.parametrize("pinned", [[0], [7, 12]])
def test_popped_fused_circuit_expectation(hq, pinned):
    """Sec. 3.1 pop, then simplify and DAG fusion, then the tensor-core
    engine: expectation values on the pinned qubits equal the oracle's on the
    full circuit."""
    circ = C.random_circuit(C.grid(4, 5), 14, seed=5, two_qubit="fsim")
    kept = hq.hq_pop(circ.n, circ.gates, pinned)
    kept = hq.hq_simplify(circ.n, kept)
    assert len(kept) < len(circ.gates)
    blocks = hq.hq_fuse(circ.n, kept, 6, method="dag", restarts=8)
    st = torch.empty(1 << circ.n, dtype=torch.complex64, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, blocks, engine="tc_f16", tc_min_k=4)
    H = [(1.0, ((pinned[0], "Z"),)), (0.5, ((pinned[-1], "X"),))]
    want = oracle.expectation(oracle.simulate(circ), H)
    assert abs(hq.hq_expectation(st, H) - want) <= 1e-5 * 1.5


def np_state(n, seed):
    """Seeded normalised Gaussian state from numpy's generator (input only;
    fast at the larger sizes)."""
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return psi / np.linalg.norm(psi)


def structured_hamiltonian(n, seed):
    """Terms of every shape the tiled kernels distinguish: diagonal strings
    with Z on low, middle and high qubits; single X and Y; XX, YY, XY, YX on
    neighbouring and distant pairs (more than four terms sharing one X mask);
    X masks of three to six qubits with Z and Y mixed in; the identity."""
    rng = C.SplitMix64(seed)

    def coeff():
        return rng.uniform() - 0.5

    H = [(0.3, ())]

    def add(c, term):
        if len({q for q, _ in term}) == len(term):
            H.append((c, term))

    for q in range(n - 1):
        H.append((coeff(), ((q, "Z"), (q + 1, "Z"))))
    for q in range(0, n, 2):
        add(coeff(), ((q, "Z"), ((q + 7) % n, "Z"), ((q + 11) % n, "Z")))
    for q in range(n):
        H.append((coeff(), ((q, "X"),)))
        if q % 3 == 0:
            H.append((coeff(), ((q, "Y"),)))
    for q in range(0, n - 1, 2):
        for a, b in (("X", "X"), ("Y", "Y"), ("X", "Y"), ("Y", "X"), ("Z", "X")):
            H.append((coeff(), ((q, a), (q + 1, b))))
    for q in range(0, n - 4, 5):
        add(coeff(), ((q, "X"), (q + 2, "Y"), (q + 4, "X"), ((q + 8) % n, "Z")))
        add(coeff(), tuple((q + j, "XY"[j % 2]) for j in range(min(6, n - q))))
    return H


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n,seed", [(13, 5), (15, 6), (19, 7), (24, 8)])
def test_expectation_structured_sums(hq, dt, n, seed):
    """Register-view tile passes (diagonal strings by a Walsh-Hadamard
    transform, X masks paired in registers or through shared memory) and the
    fallback kernels, against the oracle."""
    psi = np_state(n, 80 + n)
    H = structured_hamiltonian(n, seed)
    want = oracle.expectation(psi, H)
    st = to_dev(psi, dt)
    got = hq.hq_expectation(st, H)
    tol = 1e-12 if dt == "c128" else 1e-5 * max(1.0, sum(abs(c) for c, _ in H))
    assert abs(got - want) <= tol, (got, want)
    # each term on its own (one X-mask group: the streaming kernel), summed
    parts = sum(hq.hq_expectation(st, [t]) for t in H[:40])
    assert abs(parts - oracle.expectation(psi, H[:40])) <= tol


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_expectation_ansatz_hamiltonian_large_state(hq, dt):
    """The ansatz Hamiltonian at n = 22 (several tile passes, every X on its
    own qubit) on a random state."""
    n = 22
    psi = np_state(n, 123)
    H = C.ansatz_hamiltonian(n)
    got = hq.hq_expectation(to_dev(psi, dt), H)
    tol = 1e-12 if dt == "c128" else 1e-5 * sum(abs(c) for c, _ in H)
    assert abs(got - oracle.expectation(psi, H)) <= tol


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_expectation_single_x_with_z_strings(hq, dt):
    """Terms whose X (or Y) is one high qubit, with Z on the lane bits, on
    bits outside the pass, and on other bits of the same pass (those leave
    the register passes for the shared-memory ones); several terms per qubit
    and more single-X terms than one parameter block holds."""
    n = 21
    psi = np_state(n, 321)
    rng = C.SplitMix64(77)
    H = []
    for q in range(n - 13):  # flat bits 13..20 are qubits 0..7
        for _ in range(14):
            zs = sorted({rng.randint(0, n - 1) for _ in range(rng.randint(0, 3))} - {q})
            H.append((rng.uniform() - 0.5, ((q, "XY"[rng.randint(0, 1)]),) + tuple((z, "Z") for z in zs)))
    H.append((0.7, ((0, "X"), (1, "Z"))))      # Z on another bit of the same register pass
    H.append((0.4, ((3, "Y"), (n - 1, "Z"))))  # Z on flat bit 0 (a lane bit)
    assert len(H) > 96
    want = oracle.expectation(psi, H)
    got = hq.hq_expectation(to_dev(psi, dt), H)
    tol = 1e-12 if dt == "c128" else 1e-5 * sum(abs(c) for c, _ in H)
    assert abs(got - want) <= tol, (got, want)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("pinned", [True, False])
def test_state_upload_from_host(hq, dt, pinned):
    """hq_state_upload: pinned host memory read by the SMs, pageable memory
    through the driver; the device state equals the host bytes exactly, and
    evolving it gives the oracle's state."""
    n = 17
    psi = np_state(n, 55)
    host = torch.from_numpy(psi).to(DT[dt])
    if pinned:
        host = host.pin_memory()
    st = torch.empty(1 << n, dtype=DT[dt], device="cuda")
    hq.hq_state_upload(st, host)
    torch.cuda.synchronize()
    assert torch.equal(st.cpu(), host)
    M = C.random_unitary(2, C.SplitMix64(4))
    hq.hq_apply_blocks(st, [((3, 11), M)])
    want = oracle.apply_gate(host.numpy().astype(np.complex128), n, (3, 11), M)
    got = st.cpu().numpy().astype(np.complex128)
    tol = 1e-12 if dt == "c128" else 2e-6
    assert np.abs(got - want).max() <= tol


def test_state_upload_argument_errors(hq):
    st = torch.empty(1 << 6, dtype=torch.complex64, device="cuda")
    host = torch.zeros(1 << 6, dtype=torch.complex64)
    with pytest.raises(ValueError):
        hq.hq_state_upload(st, host[:32])
    lib = hq.load()
    assert lib.hq_state_upload(hq.ctypes.c_void_p(st.data_ptr()), None, 6, hq.HQ_C64, None) == -1
    assert lib.hq_state_upload(hq.ctypes.c_void_p(st.data_ptr()), hq.ctypes.c_void_p(host.data_ptr() + 8), 6,
                               hq.HQ_C64, None) == -13


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_expectation_low_pass_overflow_and_lane_signs(hq, dt):
    """More diagonal and low one-bit-X terms than the low pass holds (the
    rest go to the shared-memory passes), X and Y on every low qubit with Z
    on lane bits, on the other layout's lane bits and above the unit."""
    n = 16
    psi = np_state(n, 404)
    rng = C.SplitMix64(405)
    H = []
    for _ in range(110):
        zs = sorted({rng.randint(0, n - 1) for _ in range(rng.randint(1, 4))})
        H.append((rng.uniform() - 0.5, tuple((z, "Z") for z in zs)))
    for q in range(n - 11, n):  # flat bits 0..10
        for op in "XY":
            zs = sorted({rng.randint(0, n - 1) for _ in range(2)} - {q})
            H.append((rng.uniform() - 0.5, ((q, op),) + tuple((z, "Z") for z in zs)))
    want = oracle.expectation(psi, H)
    got = hq.hq_expectation(to_dev(psi, dt), H)
    tol = 1e-12 if dt == "c128" else 1e-5 * sum(abs(c) for c, _ in H)
    assert abs(got - want) <= tol, (got, want)
