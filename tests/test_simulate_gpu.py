"""hq_simulate (Sec. 4.2 simulate(circuit, initial_state)): the product state
of the Sec. 4.1 tokens, the fused blocks, and the FP64 squared norm in one
call.  On the tensor-core engines the first block computes its input from the
tokens and the last block sums the norm in its epilogue; the state must equal
the separate hq_state_init + hq_apply_blocks passes bit for bit (the same
input values reach the same kernel), and both must meet the oracle within the
complex64 bar.  The fallbacks (first or last block off the tensor cores, other
engines, complex128, no blocks) are checked the same way."""
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


def rel_l2(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


def grid_blocks(hq, n, depth, seed):
    lay = C.layout_for(n)
    circ = C.random_circuit(lay, depth, seed=seed, two_qubit="fsim")
    return circ, hq.hq_fuse(n, circ.gates, 6, method="beam", width=16, seed=seed)


TOKENS = {13: ["0" * 13, "+-01+-01+-01+", "1" * 13], 14: ["+" * 14, "-1+0" * 3 + "+-"],
          17: ["0" * 17, "+0-1" * 4 + "-"]}


@pytest.mark.parametrize("engine", ["tc_f16", "tc_bf16"])
@pytest.mark.parametrize("n", [13, 14, 17])
def test_simulate_equals_separate_passes_and_oracle(hq, engine, n):
    circ, blocks = grid_blocks(hq, n, 8, seed=n)
    assert len(blocks[0][0]) >= 4 and len(blocks[-1][0]) >= 4  # first and last on the tensor cores
    tol = 2e-5 if engine == "tc_f16" else 3e-4
    for tokens in TOKENS[n]:
        a = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        a.fill_(complex(float("nan"), 0.0))  # never read
        nrm = hq.hq_simulate(a, blocks, tokens=tokens, engine=engine, tc_min_k=4)
        b = torch.empty_like(a)
        hq.hq_state_init(b, tokens)
        hq.hq_apply_blocks(b, blocks, engine=engine, tc_min_k=4)
        torch.cuda.synchronize()
        assert torch.equal(a, b), tokens
        want = oracle.simulate(circ, tokens=tokens)
        assert rel_l2(a.cpu().numpy().astype(np.complex128), want) <= tol
        # the fused norm: FP32 sums of at most 16 squares per tile and thread,
        # FP64 beyond, within 1e-8 relative of the exact sum of the stored
        # floats (the streaming norm of the separate pass likewise)
        exact = oracle.norm2(a.cpu().numpy().astype(np.complex128))
        sep = hq.hq_expectation(b, [(1.0, ())])
        assert abs(nrm - exact) <= 1e-8 * exact, (nrm, exact)
        assert abs(sep - exact) <= 1e-8, (sep, exact)
        assert abs(nrm - 1.0) <= 2 * tol


def test_simulate_norm_of_a_non_unitary_last_block(hq):
    """The epilogue's sum is the norm of what it writes: a last block scaled by
    1.5 gives 2.25 (against the oracle's FP64 sum of the same state)."""
    n = 15
    circ, blocks = grid_blocks(hq, n, 6, seed=3)
    qs, m = blocks[-1]
    blocks = blocks[:-1] + [(qs, 1.5 * m)]
    st = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    nrm = hq.hq_simulate(st, blocks, engine="tc_f16", tc_min_k=4)
    got = st.cpu().numpy().astype(np.complex128)
    assert abs(nrm - oracle.norm2(got)) <= 1e-8 * 2.25
    assert abs(nrm - 2.25) <= 2.25 * 4e-5


@pytest.mark.parametrize("where", ["first", "last", "both"])
def test_simulate_with_blocks_off_the_tensor_cores(hq, where):
    """A first (last) block that is not a tensor-core block: the initialisation
    (the norm) runs as its own pass; the result is the same."""
    n = 14
    circ, blocks = grid_blocks(hq, n, 6, seed=5)
    rz = C.rot("Z", 0.37)
    h = C.hadamard()
    if where in ("first", "both"):
        blocks = [((2,), h)] + blocks
        circ = C.Circuit(n, [C.Gate("H", (2,), h)] + circ.gates)
    if where in ("last", "both"):
        blocks = blocks + [((5,), rz)]
        circ = C.Circuit(n, circ.gates + [C.Gate("RZ", (5,), rz)])
    tokens = "+0" * 7
    a = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    nrm = hq.hq_simulate(a, blocks, tokens=tokens, engine="tc_f16", tc_min_k=4)
    b = torch.empty_like(a)
    hq.hq_state_init(b, tokens)
    hq.hq_apply_blocks(b, blocks, engine="tc_f16", tc_min_k=4)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert abs(nrm - oracle.norm2(b.cpu().numpy().astype(np.complex128))) <= 1e-8
    assert rel_l2(a.cpu().numpy().astype(np.complex128), oracle.simulate(circ, tokens=tokens)) <= 2e-5


def _monomial_4q(seed):
    """A 4-qubit permutation with phases (one nonzero per row and column)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(16)
    m = np.zeros((16, 16), np.complex128)
    m[np.arange(16), perm] = np.exp(1j * rng.uniform(0, 2 * np.pi, 16))
    return m


def test_simulate_folds_the_norm_into_a_structured_last_block(hq):
    """A last block that the monomial kernel would take runs on the tensor
    cores inside hq_simulate so that its epilogue sums the norm: the state
    meets the oracle within the complex64 bar and the separate passes (exact
    monomial kernel) within split-precision rounding; the norm is that of
    the stored state."""
    n = 14
    circ, blocks = grid_blocks(hq, n, 6, seed=9)
    qs = (1, 4, 7, 11)
    m = _monomial_4q(9)
    s, _, _ = hq.hq_gate_structure(m)
    assert s & 2  # monomial
    blocks = blocks + [(qs, m)]
    circ = C.Circuit(n, circ.gates + [C.Gate("P", qs, m)])
    tokens = "+-" * 7
    a = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    nrm = hq.hq_simulate(a, blocks, tokens=tokens, engine="tc_f16", tc_min_k=4)
    b = torch.empty_like(a)
    hq.hq_state_init(b, tokens)
    hq.hq_apply_blocks(b, blocks, engine="tc_f16", tc_min_k=4)
    got = a.cpu().numpy().astype(np.complex128)
    sep = b.cpu().numpy().astype(np.complex128)
    assert rel_l2(got, oracle.simulate(circ, tokens=tokens)) <= 2e-5
    assert rel_l2(got, sep) <= 1e-6
    assert abs(nrm - oracle.norm2(got)) <= 1e-8 * oracle.norm2(got)
    assert abs(nrm - 1.0) <= 4e-5


@pytest.mark.parametrize("dtype,engine,tol", [(torch.complex128, "auto", 1e-12), (torch.complex128, "df", 1e-12),
                                              (torch.complex64, "auto", 2e-5), (torch.complex64, "cuda_core", 2e-5)])
def test_simulate_other_engines(hq, dtype, engine, tol):
    n = 13
    circ, blocks = grid_blocks(hq, n, 5, seed=7)
    if engine == "df":
        blocks = hq.hq_fuse(n, circ.gates, 4, method="beam", width=16)
    st = torch.empty(1 << n, dtype=dtype, device="cuda")
    nrm = hq.hq_simulate(st, blocks, tokens="-" * n, engine=engine)
    want = oracle.simulate(circ, tokens="-" * n)
    got = st.cpu().numpy().astype(np.complex128)
    if dtype == torch.complex128:
        assert np.max(np.abs(got - want)) <= tol
    else:
        assert rel_l2(got, want) <= tol
    assert abs(nrm - 1.0) <= 10 * tol


def test_simulate_without_norm_and_without_blocks(hq):
    n = 13
    st = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    assert hq.hq_simulate(st, [], tokens="+" * n, engine="tc_f16", norm=False) is None
    torch.cuda.synchronize()
    want = oracle.state_init(n, "+" * n)
    assert np.max(np.abs(st.cpu().numpy().astype(np.complex128) - want)) <= 1e-7
    assert abs(hq.hq_simulate(st, [], tokens="1" * n, engine="tc_f16") - 1.0) <= 1e-7
    circ, blocks = grid_blocks(hq, n, 4, seed=9)
    assert hq.hq_simulate(st, blocks, engine="tc_f16", tc_min_k=4, norm=False) is None
    torch.cuda.synchronize()
    assert rel_l2(st.cpu().numpy().astype(np.complex128), oracle.simulate(circ)) <= 2e-5


def test_simulate_errors(hq):
    n = 13
    st = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    with pytest.raises(hq.HQError, match="TOKEN"):
        hq.hq_simulate(st, [], tokens="0" * 12 + "x", engine="tc_f16")
    with pytest.raises(hq.HQError, match="DTYPE"):
        hq.hq_simulate(torch.empty(1 << n, dtype=torch.complex128, device="cuda"), [], engine="tc_f16")
    with pytest.raises(hq.HQError, match="QUBIT_RANGE"):
        hq.hq_simulate(st, [((13,), np.eye(2))], engine="tc_f16")
