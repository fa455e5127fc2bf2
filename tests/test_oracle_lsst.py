"""Pins of the oracle's low-stretch spanning tree (Section III-B backbone,
built by weight classes and low-diameter decompositions) and of its total
stretch, against published generator outputs, hand-worked decompositions,
the breadth-first-search definition of the shifted decomposition, graph
connectivity, and dense linear algebra.  Includes planted mistakes that the
pins must catch."""
import json
import os

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components, shortest_path

import oracle
from synth import graphs

HERE = os.path.dirname(__file__)


def _og(n, u, v, w):
    rowptr, col, val = graphs.csr_from_edges(n, np.asarray(u), np.asarray(v),
                                             np.asarray(w, dtype=np.float64))
    return oracle.extract(n, rowptr, col, val)


def _components(n, u, v):
    if len(u) == 0:
        return n
    a = coo_matrix((np.ones(len(u)), (u, v)), shape=(n, n))
    return connected_components(a, directed=False)[0]


def _random_connected(n, extra, seed, wlo=-3.0, whi=3.0):
    rng = np.random.default_rng(seed)
    # a random spanning tree plus random extra edges, weights 2^U(wlo, whi)
    perm = rng.permutation(n)
    u = [int(perm[i]) for i in range(1, n)]
    v = [int(perm[rng.integers(0, i)]) for i in range(1, n)]
    pairs = {(min(a, b), max(a, b)) for a, b in zip(u, v)}
    while len(pairs) < n - 1 + extra:
        a, b = rng.integers(0, n, 2)
        if a != b:
            pairs.add((int(min(a, b)), int(max(a, b))))
    pairs = sorted(pairs)
    u = np.array([p[0] for p in pairs])
    v = np.array([p[1] for p in pairs])
    w = 2.0 ** rng.uniform(wlo, whi, len(pairs))
    return _og(n, u, v, w)


# ---------------------------------------------------------------- generator

def test_splitmix64_published_outputs():
    """The first three outputs of SplitMix64 seeded with 0."""
    g = oracle._GOLDEN
    m = (1 << 64) - 1
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(g & m) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64((2 * g) & m) == 0x06C45D188009454F


def test_shift_distribution_geometric():
    """P(shift >= 3k) = 2^-k: binomial 5-sigma bands over 200k clusters."""
    N = 200_000
    s = np.array([oracle.lsst_shift(7, 2, 5, x) for x in range(N)])
    assert np.all(s % 3 == 0) and s.min() == 0 and s.max() <= 60
    for k in range(1, 8):
        p = 2.0 ** -k
        f = np.mean(s >= 3 * k)
        assert abs(f - p) <= 5 * np.sqrt(p * (1 - p) / N), (k, f, p)
    # different (class, level) give different draws
    s2 = np.array([oracle.lsst_shift(7, 2, 6, x) for x in range(2000)])
    assert np.mean(s2 != s[:2000]) > 0.3


def test_classes_hand_values():
    """Binary exponents: 1 = 0.5*2^1, 2 and 3 in [2,4), 4 and 7.99 in [4,8),
    8 = 0.5*2^4, 0.5 = 0.5*2^0; class = 4 - e."""
    w = np.array([1.0, 2.0, 3.0, 4.0, 0.5, 7.99, 8.0])
    assert list(oracle.lsst_classes(w)) == [3, 2, 2, 1, 4, 1, 0]


# ---------------------------------------------------------------- decomposition

def _ldd_by_definition(X, A, B, E, ew, start):
    """The decomposition by its closed form: claim round of x =
    min_u (start_u + hops(u, x)); centre = the u attaining it with the
    smallest (start_u, u); join edge = the heaviest (smallest id on equal
    weight) edge from x to a neighbour y with the same centre and claim
    round one less."""
    X = [int(x) for x in X]
    idx = {x: i for i, x in enumerate(X)}
    k = len(X)
    a = np.array([idx[int(x)] for x in A])
    b = np.array([idx[int(x)] for x in B])
    adj = coo_matrix((np.ones(len(a)), (a, b)), shape=(k, k)).tocsr()
    hops = shortest_path(adj, directed=False, unweighted=True)
    centre, when, via = {}, {}, {}
    for j, x in enumerate(X):
        best = None
        for i, u in enumerate(X):
            if np.isinf(hops[i, j]):
                continue
            key = (start[u] + int(hops[i, j]), start[u], u)
            if best is None or key < best:
                best = key
        when[x] = best[0]
        centre[x] = best[2]
    for x in X:
        if centre[x] == x:
            continue
        cand = []
        for p, q, e in zip(A, B, E):
            p, q, e = int(p), int(q), int(e)
            for s, t in ((p, q), (q, p)):
                if s == x and centre[t] == centre[x] and when[t] == when[x] - 1:
                    cand.append((-float(ew[e]), e))
        via[x] = min(cand)[1]
    return centre, when, via


def test_ldd_hand_path():
    """Path 0-1-2-3-4, unit weights, starts (2, 1, 3, 0, 3): round 0 makes 3
    a centre; round 1: 2 and 4 join 3 (edges 2 and 3), then 1 starts; round
    2: 0 joins 1 through edge 0."""
    with open(os.path.join(HERE, "golden", "lsst_ldd_hand.json")) as f:
        case = json.load(f)
    for c in case["cases"]:
        start = {int(k): v for k, v in c["start"].items()}
        centre, when, via = oracle.lsst_ldd(c["X"], c["A"], c["B"], c["E"],
                                            np.array(c["w"]), start)
        assert centre == {int(k): v for k, v in c["centre"].items()}, c["name"]
        assert when == {int(k): v for k, v in c["when"].items()}, c["name"]
        assert via == {int(k): v for k, v in c["via"].items()}, c["name"]


@pytest.mark.parametrize("seed", range(6))
def test_ldd_matches_definition(seed):
    rng = np.random.default_rng(100 + seed)
    k = 40
    X = sorted(rng.choice(1000, k, replace=False).tolist())
    # connected-ish random cluster graph with repeated pairs
    A, B = [], []
    for i in range(1, k):
        A.append(X[i]); B.append(X[rng.integers(0, i)])
    for _ in range(30):
        i, j = rng.integers(0, k, 2)
        if i != j:
            A.append(X[i]); B.append(X[j])
    for _ in range(10):     # repeated pairs
        t = rng.integers(0, len(A))
        A.append(A[t]); B.append(B[t])
    E = list(range(len(A)))
    # small weight set so that ties on weight occur
    ew = rng.choice([1.0, 2.0, 3.0], len(A))
    start = {x: int(rng.integers(0, 7)) for x in X}
    got = oracle.lsst_ldd(X, A, B, E, ew, start)
    want = _ldd_by_definition(X, A, B, E, ew, start)
    assert got[0] == want[0]
    assert got[1] == want[1]
    assert got[2] == want[2]


def test_ldd_planted_mistake_caught():
    """A decomposition that prefers the largest centre id on equal starts
    (planted by renaming x -> 8 - x around the oracle's) fails the
    definition check on a 3 x 3 grid where the centre of the middle cluster
    is decided by that tie."""
    X = list(range(9))
    A = [0, 1, 3, 4, 6, 7, 0, 3, 1, 4, 2, 5]
    B = [1, 2, 4, 5, 7, 8, 3, 6, 4, 7, 5, 8]
    E = list(range(len(A)))
    ew = np.ones(len(A))
    start = {x: 0 for x in X}
    start[4] = 1
    want = _ldd_by_definition(X, A, B, E, ew, start)
    assert want[0][4] == 1
    assert oracle.lsst_ldd(X, A, B, E, ew, start)[0] == want[0]

    def ldd_largest_first(X, A, B, E, ew, start):
        c, w, v = oracle.lsst_ldd([8 - x for x in X], [8 - a for a in A], [8 - b for b in B],
                                  E, ew, {8 - x: s for x, s in start.items()})
        return ({8 - x: 8 - cc for x, cc in c.items()}, {8 - x: t for x, t in w.items()},
                {8 - x: e for x, e in v.items()})
    assert ldd_largest_first(X, A, B, E, ew, start)[0] != want[0]


# ---------------------------------------------------------------- the tree

def _check_spanning_and_classes(og, t):
    n = og.n
    te = np.flatnonzero(t)
    assert te.shape[0] == n - 1
    assert _components(n, og.eu[te], og.ev[te]) == 1
    cls = oracle.lsst_classes(og.ew)
    for c in range(int(cls.max()) + 1):
        sub = np.flatnonzero(cls <= c)
        comps = _components(n, og.eu[sub], og.ev[sub])
        tc = np.flatnonzero((t != 0) & (cls <= c))
        # the tree's edges of classes <= c span every component of G_{<=c}
        assert tc.shape[0] == n - comps, (c, tc.shape[0], n - comps)


@pytest.mark.parametrize("seed", range(4))
def test_lsst_spanning_tree_class_forests(seed):
    og = _random_connected(300, 500, seed)
    t = oracle.low_stretch_tree(og, seed=11 + seed)
    _check_spanning_and_classes(og, t)


def test_lsst_planted_class_order_caught(monkeypatch):
    """Lightest class first breaks the class-forest property."""
    og = _random_connected(200, 400, 3)
    real = oracle.lsst_classes
    monkeypatch.setattr(oracle, "lsst_classes", lambda w: real(w).max() - real(w))
    bad = oracle.low_stretch_tree(og, seed=1)
    monkeypatch.setattr(oracle, "lsst_classes", real)
    with pytest.raises(AssertionError):
        _check_spanning_and_classes(og, bad)
    _check_spanning_and_classes(og, oracle.low_stretch_tree(og, seed=1))


def test_lsst_of_a_tree_is_the_tree():
    rng = np.random.default_rng(2)
    n = 120
    u = np.arange(1, n)
    v = np.array([rng.integers(0, i) for i in range(1, n)])
    og = _og(n, np.minimum(u, v), np.maximum(u, v), 2.0 ** rng.uniform(-4, 4, n - 1))
    assert np.all(oracle.low_stretch_tree(og, seed=3) == 1)


def test_lsst_heavy_path_with_light_chords():
    """A path of weight 1000 plus chords of weight 1: the tree is the path."""
    n = 60
    rng = np.random.default_rng(4)
    pairs = {(i, i + 1): 1000.0 for i in range(n - 1)}
    while len(pairs) < n - 1 + 80:
        a, b = sorted(rng.integers(0, n, 2))
        if b > a + 1:
            pairs[(int(a), int(b))] = 1.0
    keys = sorted(pairs)
    u = np.array([k[0] for k in keys]); v = np.array([k[1] for k in keys])
    w = np.array([pairs[k] for k in keys])
    og = _og(n, u, v, w)
    t = oracle.low_stretch_tree(og, seed=9)
    assert np.all((t != 0) == (og.ew == 1000.0))


def test_lsst_deterministic_and_seeded():
    og = oracle.from_graph(graphs.grid((24, 24)))
    a = oracle.low_stretch_tree(og, seed=1)
    b = oracle.low_stretch_tree(og, seed=1)
    c = oracle.low_stretch_tree(og, seed=2)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


# ---------------------------------------------------------------- stretch

@pytest.mark.parametrize("kind", ["mst", "lsst"])
def test_total_stretch_is_trace(kind):
    """st_T(G) = Tr(L_T^+ L_G) for a spanning tree T of G (each edge's
    stretch is w_e b_e^T L_T^+ b_e); tree edges have stretch 1.  The trace
    is taken with row and column 0 removed from both Laplacians (b_e sums
    to zero, so b^T L_T^+ b is the grounded quadratic form), by a dense
    solve."""
    og = _random_connected(70, 120, 8)
    t = oracle.mst(og) if kind == "mst" else oracle.low_stretch_tree(og, seed=4)
    tot, st = oracle.total_stretch(og, t)
    n = og.n

    def lap(mask):
        L = np.zeros((n, n))
        for e in np.flatnonzero(mask):
            p, q, w = og.eu[e], og.ev[e], og.ew[e]
            L[p, p] += w; L[q, q] += w; L[p, q] -= w; L[q, p] -= w
        return L
    LT = lap(t != 0)
    LG = lap(np.ones(og.m, bool))
    tr = np.trace(np.linalg.solve(LT[1:, 1:], LG[1:, 1:]))
    assert abs(tot - tr) <= 1e-9 * tr
    assert np.allclose(st[t != 0], 1.0, rtol=0, atol=1e-12)


def test_cycle_total_stretch():
    """Unit cycle of n: any spanning tree leaves one edge of stretch n - 1."""
    n = 50
    u = np.arange(n); v = (u + 1) % n
    og = _og(n, np.minimum(u, v), np.maximum(u, v), np.ones(n))
    t = oracle.low_stretch_tree(og, seed=5)
    tot, _ = oracle.total_stretch(og, t)
    assert t.sum() == n - 1
    assert abs(tot - 2 * (n - 1)) <= 1e-9


def test_lsst_beats_mst_stretch_on_unit_grid():
    """On a unit-weight mesh the id-ordered maximum-weight tree is a comb of
    stretch O(side) per edge; the low-stretch tree stays far below it."""
    og = oracle.from_graph(graphs.grid((48, 48)))
    st_l, _ = oracle.total_stretch(og, oracle.low_stretch_tree(og, seed=1))
    st_m, _ = oracle.total_stretch(og, oracle.mst(og))
    assert st_l < 0.5 * st_m
