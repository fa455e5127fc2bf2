"""Pins of the oracle's spectral partitioner (Sec. V-F): inverse power
iterations converge to the Fiedler vector that the mathematics fixes.

* path graph P_n, unit weights: the Fiedler vector is cos(pi (i + 1/2) / n)
  with eigenvalue 2 - 2 cos(pi / n), and the sign cut halves the path;
* two cliques joined by one light edge: the sign cut separates the cliques;
* small random graphs: the dense eigensolver's second eigenvector.
Planted mistakes (no projection against the all-ones vector, forward
instead of inverse iterations) fail a pin."""
import numpy as np
import pytest

import oracle
from synth import graphs, rng
from tests.helpers import dense_lap, tiny_graph


def _og(n, u, v, w, D=0.0):
    rp, col, val = graphs.csr_from_edges(n, np.asarray(u), np.asarray(v), np.asarray(w, float), D)
    return oracle.from_graph(graphs.Graph("g", n, rp, col, val))


def test_path_graph_closed_form():
    n = 40
    og = _og(n, np.arange(n - 1), np.arange(1, n), np.ones(n - 1))
    ot = oracle.build_tree(og)
    u, side, lam, _ = oracle.fiedler(og, ot, None, rng.normal(1, 1, n), 60, 1e-13)
    v = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    v /= np.linalg.norm(v)
    assert abs(abs(u @ v) - 1.0) <= 1e-9
    assert lam == pytest.approx(2.0 - 2.0 * np.cos(np.pi / n), rel=1e-9)
    assert side.sum() == n // 2
    assert len(set(side[: n // 2])) == 1 and len(set(side[n // 2:])) == 1


def test_two_cliques_are_separated():
    k = 12
    us, vs = [], []
    for base in (0, k):
        for a in range(k):
            for b in range(a + 1, k):
                us.append(base + a)
                vs.append(base + b)
    w = list(1.0 + rng.uniform(3, 1, len(us)))
    us.append(k - 1)
    vs.append(k)
    w.append(0.01)
    og = _og(2 * k, us, vs, w)
    ot = oracle.build_tree(og)
    in_s = ot.in_tree.copy()
    in_s[np.flatnonzero(in_s == 0)[::2]] = 1
    u, side, lam, _ = oracle.fiedler(og, ot, in_s, rng.normal(3, 2, 2 * k), 8, 1e-10,
                                     inner_tol=1e-13, inner_maxit=500)
    assert len(set(side[:k])) == 1 and len(set(side[k:])) == 1 and side[0] != side[k]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_matches_dense_second_eigenvector(seed):
    g = tiny_graph(30, 25, seed)
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    L = dense_lap(g.n, og.eu, og.ev, og.ew)
    lam, V = np.linalg.eigh(L)
    gap = lam[2] / lam[1]
    its = int(np.ceil(np.log(1e-10) / np.log(1.0 / gap))) + 2
    u, side, lq, _ = oracle.fiedler(og, ot, None, rng.normal(seed, 4, g.n), its, 1e-13)
    assert abs(abs(u @ V[:, 1]) - 1.0) <= 1e-8
    assert lq == pytest.approx(lam[1], rel=1e-8)


def test_planted_mistakes_fail_a_pin():
    n = 40
    og = _og(n, np.arange(n - 1), np.arange(1, n), np.ones(n - 1))
    ot = oracle.build_tree(og)
    v = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    v /= np.linalg.norm(v)
    x0 = rng.normal(1, 1, n) + 5.0                   # a large constant component

    def no_projection(x, its):
        x = x / np.linalg.norm(x)
        for _ in range(its):
            y, *_ = oracle.pcg(og, ot, None, x, 1e-13, 5000)
            x = y / np.linalg.norm(y)
        return x

    def forward(x, its):
        L = dense_lap(n, og.eu, og.ev, og.ew)
        x = x - x.mean()
        for _ in range(its):
            x = L @ x
            x -= x.mean()
            x /= np.linalg.norm(x)
        return x
    for fn in (no_projection, forward):
        u = fn(x0.copy(), 60)
        assert not (abs(abs(u @ v) - 1.0) <= 1e-6), fn.__name__     # NaN fails the pin too
