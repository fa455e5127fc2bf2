"""Pins of the oracle's similarity check (Sec. IV-D step 6, endpoint-conflict
reading): a hand-worked case, and the two properties that fix the greedy
result uniquely for a strict priority order -- the kept edges form a
matching, and every selected edge that was not kept has an endpoint on a
kept edge of higher priority (so no kept edge could have been rejected and
no rejected edge could have been kept).  Planted mistakes (ascending heat
order, no conflict test) fail a pin."""
import json
import os

import numpy as np
import pytest

import oracle
from synth import graphs, rng
from tests.helpers import tiny_graph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "similarity_hand.json")


def _hand():
    d = json.load(open(GOLDEN))
    edges = d["tree_edges"] + d["off_edges"]
    u = np.array([min(a, b) for a, b in edges])
    v = np.array([max(a, b) for a, b in edges])
    rp, col, val = graphs.csr_from_edges(d["n"], u, v, np.ones(len(edges)), 0.0)
    og = oracle.from_graph(graphs.Graph("hand", d["n"], rp, col, val))
    key = {(int(a), int(b)): e for e, (a, b) in enumerate(zip(og.eu, og.ev))}
    tree = set(key[(min(a, b), max(a, b))] for a, b in d["tree_edges"])
    off = np.array(sorted(e for e in range(og.m) if e not in tree), dtype=np.int64)
    hv = np.array([d["heat"][f"{og.eu[e]}-{og.ev[e]}"] for e in off])
    return d, og, key, off, hv


def test_hand_worked_cases():
    d, og, key, off, hv = _hand()
    for c in d["cases"]:
        want = sorted(key[(a, b)] for a, b in c["kept"])
        got = oracle.similarity_check(og, hv, off, c["theta"], c["cap"])
        assert list(got) == want, c
    # without the check every selected edge passes (the check is what removes them)
    assert len(oracle.filter_edges(hv, off, 0.1)) == 7


def _priority(hv, off):
    """rank of each off-edge position: 0 = visited first"""
    order = np.lexsort((off, -hv))
    rank = np.empty_like(order)
    rank[order] = np.arange(order.shape[0])
    return rank


def _greedy_properties(og, hv, off, theta, kept):
    """The matching and domination properties; returns the violations."""
    bad = []
    pos = {int(e): i for i, e in enumerate(off)}
    rank = _priority(hv, off)
    thr = theta * hv.max()
    ends = {}
    for e in kept:
        for x in (int(og.eu[e]), int(og.ev[e])):
            if x in ends:
                bad.append(("not a matching", int(e)))
            ends[x] = int(e)
    keptset = set(int(e) for e in kept)
    for i, e in enumerate(off):
        if hv[i] < thr or int(e) in keptset:
            continue
        blockers = [ends[x] for x in (int(og.eu[e]), int(og.ev[e])) if x in ends]
        if not any(rank[pos[b]] < rank[i] for b in blockers):
            bad.append(("rejected without a better kept neighbour", int(e)))
    for e in kept:
        if hv[pos[int(e)]] < thr:
            bad.append(("below threshold", int(e)))
    return bad


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_greedy_characterisation_on_random_graphs(seed):
    g = tiny_graph(60, 140, seed)
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    off = np.flatnonzero(ot.in_tree == 0).astype(np.int64)
    # integer heats: many ties, so the id order matters
    hv = (rng.raw64(seed, 77, 0, off.shape[0]) % np.uint64(7)).astype(np.float64)
    for theta in (0.0, 0.3, 0.9):
        kept = oracle.similarity_check(og, hv, off, theta)
        assert _greedy_properties(og, hv, off, theta, kept) == []
        assert len(kept) > 0
        # cap: the first kept edges in priority order
        rank = _priority(hv, off)
        pos = {int(e): i for i, e in enumerate(off)}
        by_rank = sorted(kept, key=lambda e: rank[pos[int(e)]])
        for cap in (1, 3):
            assert list(oracle.similarity_check(og, hv, off, theta, cap)) == sorted(by_rank[:cap])


def test_planted_mistakes_fail_a_pin():
    d, og, key, off, hv = _hand()

    def ascending(og_, hv_, off_, theta, cap=0):
        return oracle.similarity_check(og_, -hv_ + hv_.max() + 1.0, off_, 0.0, cap)

    def no_conflicts(og_, hv_, off_, theta, cap=0):
        return oracle.filter_edges(hv_, off_, theta, cap)

    for fn in (ascending, no_conflicts):
        bad = 0
        for c in d["cases"]:
            want = sorted(key[(a, b)] for a, b in c["kept"])
            bad += list(fn(og, hv, off, c["theta"], c["cap"])) != want
        assert bad > 0, fn.__name__
    # the tie at heat 9 (0-3 before 1-3 by id) decides the hand case: taking
    # 1-3 first would keep {1-3, 2-4}, which the golden set rejects
    assert key[(0, 3)] < key[(1, 3)]
