"""Batched persistent runs (hq_batch_*): every circuit of a mixed-size batch
against the oracle, for several tile shapes, across graph replays."""
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


def small_batch():
    cs = C.config_batch(40, seed=3, n_range=(3, 17), depth_range=(2, 14))
    cs.append(C.Circuit(5, []))  # no gates: |0..0>
    cs.append(C.random_circuit(C.layout_for(1), 3, 1, "cz"))  # one qubit
    return cs


def rel_l2(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


@pytest.mark.parametrize("cfg", [(0, 0, 0, 0), (8, 3, 0, 1), (11, 5, 2, 0), (13, 7, 0, 1), (6, 1, 1, 0),
                                 (12, 6, 0, 0, 1), (12, 6, 0, 1, 3), (13, 7, 0, 0, 3), (8, 3, 0, 0, 3)])
def test_batch_matches_oracle(hq, cfg):
    """cfg = (tile_bits, max_high, ctas_per_sm, small_first[, fuse_k])."""
    cs = small_batch()
    b = hq.Batch(cs, None, *cfg)
    for rep in range(2):  # the second replay rebuilds every state from |0..0>
        b.run()
        lat, span = b.latencies()
        assert np.all(lat > 0) and np.all(lat <= span + 1e-3)
        for c, st in zip(cs, b.states):
            want = oracle.simulate(c)
            got = st.cpu().numpy().astype(np.complex128)
            assert rel_l2(got, want) <= 2e-5 * max(1, len(c.gates) / 1000), (c.n, len(c.gates), cfg)
    b.close()


def test_batch_argument_errors(hq):
    wide = C.Circuit(6, [C.Gate("U3", (0, 1, 2), C.random_unitary(3, C.SplitMix64(1)))])
    with pytest.raises(hq.HQError, match="K_TOO_LARGE"):
        hq.Batch([wide])
    with pytest.raises(hq.HQError, match="ARG"):
        hq.Batch([C.config_small(0)], None, 14, 6, 0)
    with pytest.raises(hq.HQError, match="ARG"):
        hq.Batch([C.config_small(0)], None, 12, 6, 0, 0, 4)  # in-pass fusion wider than 3 qubits


@pytest.mark.slow
def test_serving_load_512_circuits(hq):
    """512 circuits, n ~ U{10..24}, depth ~ U{8..32}: every circuit of up to
    20 qubits and four of 22 or more against the oracle, every state's norm on
    the GPU."""
    cs = C.config_batch(512, seed=0)
    b = hq.Batch(cs)
    b.run()
    lat, span = b.latencies()
    assert np.all(lat > 0)
    small = [i for i, c in enumerate(cs) if c.n <= 20]
    big = [i for i, c in enumerate(cs) if c.n >= 22][:4]
    assert len(small) > 300
    for i in small + big:
        want = oracle.simulate(cs[i])
        got = b.states[i].cpu().numpy().astype(np.complex128)
        assert rel_l2(got, want) <= 2e-5 * max(1, len(cs[i].gates) / 1000)
    for i, st in enumerate(b.states):
        # relative L2 bound on the state => | ||psi|| - 1 | <= the same bound
        nrm = hq.hq_expectation(st, [(1.0, ())]) ** 0.5
        assert abs(nrm - 1) <= 2e-5 * max(1, len(cs[i].gates) / 1000)
    b.close()


def test_autotuner_picks_a_candidate(hq, tmp_path):
    """The tuner times every (tile shape, fusion width) candidate, returns the
    fastest, caches it, and its choice runs the batch to the oracle's states."""
    from paper_2111_06868_gb300 import autotune

    cs = small_batch()[:12]
    cands = autotune.candidates(0, tiles=[(12, 6, 0), (11, 5, 0)], widths=[1, 2, 3])
    best, timings = autotune.tune(cs, cands=cands, reps=2, cache_path=str(tmp_path / "a.json"))
    assert best in cands and len(timings) == len(cands)
    assert timings[str(best)] == min(timings.values())
    again, _ = autotune.tune(cs, cands=cands, reps=2, cache_path=str(tmp_path / "a.json"))
    assert again == best
    p50, _ = autotune.tune(cs, cands=cands, reps=2, cache_path=str(tmp_path / "a.json"), objective="p50")
    assert p50 in cands
    b = hq.Batch(cs, None, *best)
    b.run()
    b.latencies()
    for c, st in zip(cs, b.states):
        assert rel_l2(st.cpu().numpy().astype(np.complex128), oracle.simulate(c)) <= 2e-5
    b.close()
