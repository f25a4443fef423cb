"""Host logic of the tile-pass engine (hq_plan_passes): every pass holds a
13-bit tile containing bits 0..6, applies at most two blocks whose targets lie
in the tile, only permutes qubits among the tile's own positions (in-place
update), reorders only blocks with disjoint targets, and ends in the caller's
layout.  Replaying the plan in complex128 (bit permutations + the oracle's
gate application) reproduces the oracle's state."""
import numpy as np
import pytest

import oracle
from paper_2111_06868_gb300 import circuits as C
from paper_2111_06868_gb300 import hq


@pytest.fixture(scope="module")
def lib():
    from paper_2111_06868_gb300 import build

    build.build()
    hq.load()
    return hq


def permute_bits(psi, n, mapping):
    """psi'[i'] = psi[i] where bit x of i moves to bit mapping[x]."""
    t = psi.reshape([2] * n)  # axis a <-> bit n-1-a
    src_axes = [None] * n
    for x in range(n):
        src_axes[n - 1 - mapping[x]] = n - 1 - x
    return np.ascontiguousarray(np.transpose(t, src_axes)).reshape(-1)


def replay(n, blocks, plan, psi):
    pos = list(range(n))  # logical bit -> physical bit
    for p in plan:
        slots, dest = p["slots"], p["dest"]
        assert slots == sorted(slots) and len(set(slots)) == 13 and set(range(7)) <= set(slots)
        assert sorted(dest) == slots, "qubits move only among the tile's positions"
        assert len(p["gates"]) <= 2
        for gi in p["gates"]:
            qs, m = blocks[gi]
            phys = [pos[n - 1 - q] for q in qs]
            assert set(phys) <= set(slots), "targets inside the tile"
            oracle.apply_gate(psi, n, [n - 1 - x for x in phys], m)
        mapping = list(range(n))
        for s, d in zip(slots, dest):
            mapping[s] = d
        psi = permute_bits(psi, n, mapping)
        inv = {s: d for s, d in zip(slots, dest)}
        pos = [inv.get(x, x) for x in pos]
    assert pos == list(range(n)), "caller's layout restored"
    return psi


def check_order(n, blocks, plan):
    order = [g for p in plan for g in p["gates"]]
    assert sorted(order) == list(range(len(blocks)))
    bits = [set(q for q in qs) for qs, _ in blocks]
    for a in range(len(order)):
        for b in range(a + 1, len(order)):
            if order[a] > order[b]:  # b moved ahead of a: they must commute
                assert not (bits[order[a]] & bits[order[b]])


@pytest.mark.parametrize("n,kmax,seed", [(14, 6, 1), (15, 5, 2), (16, 6, 3), (16, 4, 4), (17, 6, 5)])
def test_plan_replays_to_oracle_state(lib, n, kmax, seed):
    circ = C.random_circuit(C.layout_for(n), 12, seed=seed, two_qubit="fsim")
    blocks = lib.hq_fuse(n, circ.gates, kmax)
    for max_blocks in (1, 2):
        plan = lib.hq_plan_passes(n, blocks, max_blocks)
        check_order(n, blocks, plan)
        psi0 = oracle.state_init(n)
        want = psi0.copy()
        for qs, m in blocks:
            oracle.apply_gate(want, n, list(qs), m)
        got = replay(n, blocks, plan, psi0.copy())
        assert np.max(np.abs(got - want)) <= 1e-12


def test_plan_structure_on_the_30_qubit_grid_circuit(lib):
    """Structure only (no state): the 30-qubit grid circuit's 61 blocks."""
    circ = C.config_n30(0)
    blocks = lib.hq_fuse(30, circ.gates, 6)
    plan = lib.hq_plan_passes(30, blocks, 2)
    check_order(30, blocks, plan)
    pos = list(range(30))
    for p in plan:
        for gi in p["gates"]:
            assert {pos[29 - q] for q in blocks[gi][0]} <= set(p["slots"])
        inv = dict(zip(p["slots"], p["dest"]))
        pos = [inv.get(x, x) for x in pos]
    assert pos == list(range(30))
    assert len(plan) < len(blocks)


def test_plan_rejects_bad_arguments(lib):
    blocks = [((0, 1), np.eye(4))]
    with pytest.raises(hq.HQError):
        lib.hq_plan_passes(13, blocks, 2)
    with pytest.raises(hq.HQError):
        lib.hq_plan_passes(14, blocks, 3)
    with pytest.raises(hq.HQError):
        lib.hq_plan_passes(14, [((0, 0), np.eye(4))], 2)
