"""hq_expectation_static: the allocation-free expectation entry point.

Some callers cannot allocate device memory at the point of the call (all
memory handed to their own pool, allocator calls forbidden in a serving loop,
or another component capturing device work).  This file checks, through the C
ABI, that the static-scratch variant returns what hq_expectation returns and
what the CPU oracle computes on a copy of the same state, on two calls in a
row (the scratch keeps the previous call's contents); that it takes no
allocation (an injected allocation failure is still pending after it); and
that it refuses sums beyond its stated limit.  It is collected last on
purpose and also passes when run alone in a fresh process.
"""
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


def seeded_state(n, seed, dtype):
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    return torch.from_numpy(psi).to(dtype).cuda()


def mixed_sum(n, seed):
    rng = C.SplitMix64(seed)
    H = [(1.0, ())]
    for _ in range(20):
        L = rng.randint(1, min(4, n))
        qs = []
        while len(qs) < L:
            q = rng.randint(0, n - 1)
            if q not in qs:
                qs.append(q)
        H.append((rng.uniform() - 0.5, tuple((q, "XYZ"[rng.randint(0, 2)]) for q in qs)))
    return H


# complex128: 1e-12; complex64: the library's expectation bar, 1e-5 x sum |coeff|
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 1e-5)])
def test_static_matches_allocating_entry_point_and_oracle_twice(hq, dtype, tol):
    # two different calls in a row: the second must not see the first's partial sums
    for n, seed in ((18, 1), (11, 2)):
        st = seeded_state(n, seed, dtype)
        H = mixed_sum(n, 10 + seed)
        scale = sum(abs(c) for c, _ in H)
        want = oracle.expectation(st.cpu().numpy().astype(np.complex128), H)
        got = hq.hq_expectation_static(st, H)
        assert abs(got - want) <= tol * scale, (n, got, want)
        assert abs(got - hq.hq_expectation(st, H)) <= tol * scale


def test_static_takes_no_allocation(hq):
    """With one scratch-allocation failure injected, the static entry point
    still succeeds, and the failure is left for the next allocating call."""
    n = 16
    st = seeded_state(n, 9, torch.complex128)
    H = mixed_sum(n, 21)
    want = oracle.expectation(st.cpu().numpy(), H)
    hq.hq_test_fail_next_allocs(1)
    try:
        got = hq.hq_expectation_static(st, H)
        with pytest.raises(hq.HQError) as e:
            hq.hq_expectation(st, H)
        assert e.value.name == "HQ_ERR_ALLOC"
    finally:
        hq.hq_test_fail_next_allocs(0)
    assert abs(got - want) <= 1e-12 * sum(abs(c) for c, _ in H)


def test_static_ansatz_hamiltonian(hq):
    n = 20
    st = seeded_state(n, 5, torch.complex64)
    H = C.ansatz_hamiltonian(n)
    a = hq.hq_expectation_static(st, H)
    b = hq.hq_expectation_static(st, H)
    want = oracle.expectation(st.cpu().numpy().astype(np.complex128), H)
    assert abs(a - want) <= 1e-5 * sum(abs(c) for c, _ in H)
    assert a == b


def test_static_rejects_too_many_groups(hq):
    n = 12
    st = seeded_state(n, 3, torch.complex128)
    # 65 distinct X masks -> 65 groups, one more than the static scratch holds
    H = [(0.1, tuple((q, "X") for q in range(n) if (m >> q) & 1)) for m in range(1, 66)]
    with pytest.raises(hq.HQError, match="CAPACITY"):
        hq.hq_expectation_static(st, H)
    # still usable afterwards
    assert abs(hq.hq_expectation_static(st, [(1.0, ())]) - 1.0) <= 1e-12
