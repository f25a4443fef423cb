"""Tile-pass engine (HQ_ENGINE_TC_PASS): fused blocks applied two per trip
through HBM with in-place qubit relayouts, against the oracle.  Same bar as
the per-block tensor-core engine (FP16 hi+lo, relative L2 <= 2e-5 per 1000
unfused gates)."""
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


def run(hq, n, blocks, psi):
    st = torch.from_numpy(psi).to(torch.complex64).cuda()
    hq.hq_apply_blocks(st, blocks, engine="tc_pass")
    torch.cuda.synchronize()
    return st.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("n,kmax,depth,seed", [(14, 6, 10, 1), (16, 6, 14, 2), (17, 5, 12, 3), (18, 4, 10, 4),
                                              (20, 6, 16, 5), (21, 6, 12, 6)])
def test_circuit_matches_oracle(hq, n, kmax, depth, seed):
    circ = C.random_circuit(C.layout_for(n), depth, seed=seed, two_qubit="fsim")
    blocks = hq.hq_fuse(n, circ.gates, kmax)
    rng = np.random.default_rng(seed)  # input only
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    want = psi.copy()
    for qs, m in blocks:
        oracle.apply_gate(want, n, list(qs), m)
    got = run(hq, n, blocks, psi)
    assert rel_l2(got, want) <= 2e-5 * max(1, len(circ.gates) / 1000), rel_l2(got, want)
    assert len(hq.hq_plan_passes(n, blocks)) < len(blocks) + 4


@pytest.mark.parametrize("targets", [[0, 1, 2, 3, 4, 5], [13, 12, 11, 10, 9, 8], [1, 3, 5, 7, 9, 11],
                                     [15, 0, 7, 3, 12, 9], [2, 6], [14]])
def test_single_and_paired_blocks_any_position(hq, targets):
    """One or two blocks on low, high, interleaved and narrow target sets
    (both thread mappings, widened blocks, tensor-map and bulk tile loads)."""
    n = 16
    rng = C.SplitMix64(len(targets) * 7 + targets[0])
    k = len(targets)
    b1 = (targets, C.random_unitary(k, rng))
    b2 = (targets[::-1], C.random_unitary(k, rng))
    for blocks in ([b1], [b1, b2]):
        r = np.random.default_rng(11)  # input only
        psi = r.standard_normal(1 << n) + 1j * r.standard_normal(1 << n)
        psi /= np.linalg.norm(psi)
        want = psi.copy()
        for qs, m in blocks:
            oracle.apply_gate(want, n, list(qs), m)
        got = run(hq, n, blocks, psi)
        assert rel_l2(got, want) <= 2e-6, (targets, len(blocks), rel_l2(got, want))


def test_sparse_basis_state(hq):
    """|0..0>: most groups all-zero in the first blocks (scale-1 path)."""
    n = 18
    circ = C.random_circuit(C.layout_for(n), 8, seed=9, two_qubit="fsim")
    blocks = hq.hq_fuse(n, circ.gates, 6)
    st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, blocks, engine="tc_pass")
    want = oracle.simulate(circ)
    assert rel_l2(st.cpu().numpy().astype(np.complex128), want) <= 2e-5


def test_small_n_falls_back_and_complex128_is_refused(hq):
    n = 13
    circ = C.random_circuit(C.layout_for(n), 6, seed=2, two_qubit="fsim")
    blocks = hq.hq_fuse(n, circ.gates, 6)
    st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    hq.hq_state_init(st)
    hq.hq_apply_blocks(st, blocks, engine="tc_pass")
    assert rel_l2(st.cpu().numpy().astype(np.complex128), oracle.simulate(circ)) <= 2e-5
    st2 = torch.zeros(1 << 14, dtype=torch.complex128, device="cuda")
    with pytest.raises(hq.HQError):
        hq.hq_apply_blocks(st2, [((0, 1), np.eye(4))], engine="tc_pass")
