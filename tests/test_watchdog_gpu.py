"""Bounded device-side waits, exercised on the GPU without a fault.

The batch runner's scheduler (warp 0 of every CTA of one persistent launch)
searches for a tile it may run and gives up when it has found none for a set
time, raising the device error flag instead of waiting forever.  A test hook
shortens that limit to 1 microsecond: the CTAs that find no tile while the
first pass of a multi-pass circuit is still running then give up, the kernel
ends, and hq_batch_latencies reports HQ_ERR_TIMEOUT.  With the limit restored
the next replay of the same graph gives the oracle's states, and the context
stays usable for every other entry point."""
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
    yield _hq
    _hq.hq_test_batch_wait_limit_ns(0)


def rel_l2(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


def test_scheduler_wait_runs_out_then_recovers(hq):
    # 16- to 18-qubit circuits on 12-bit tiles with 6 high bits: a first pass
    # that fills its high bits has 2^(n - 12) tiles, far fewer than the
    # launch's CTAs (several per SM), so most CTAs find nothing to run while
    # the first passes are in flight
    cs = [C.random_circuit(C.layout_for(n), 10, seed, "cz") for n, seed in ((16, 1), (18, 2), (17, 3))]
    want = [oracle.simulate(c) for c in cs]
    b = hq.Batch(cs, None, 12, 6, 0, 0)
    try:
        hq.hq_test_batch_wait_limit_ns(1000)
        b.run()
        with pytest.raises(hq.HQError) as e:
            b.latencies()
        assert e.value.name == "HQ_ERR_TIMEOUT"
    finally:
        hq.hq_test_batch_wait_limit_ns(0)
    # the flag was read and cleared: the same graph now runs to the end
    for _ in range(2):
        b.run()
        lat, span = b.latencies()
        assert np.all(lat > 0) and np.all(lat <= span + 1e-3)
        for c, st, w in zip(cs, b.states, want):
            assert rel_l2(st.cpu().numpy().astype(np.complex128), w) <= 2e-5
    b.close()
    # other entry points are unaffected
    st = torch.empty(1 << 10, dtype=torch.complex128, device="cuda")
    hq.hq_state_init(st, "+")
    assert abs(hq.hq_expectation(st, [(1.0, ((3, "X"),))]) - 1.0) <= 1e-12


def test_limit_argument_round_trip(hq):
    hq.hq_test_batch_wait_limit_ns(5_000_000_000)
    hq.hq_test_batch_wait_limit_ns(0)
    c = C.config_small(0)
    b = hq.Batch([c], None, 10, 4, 0, 0)
    b.run()
    b.latencies()
    assert rel_l2(b.states[0].cpu().numpy().astype(np.complex128), oracle.simulate(c)) <= 2e-5
    b.close()
