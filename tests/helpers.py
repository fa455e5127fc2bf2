"""Small shared helpers for the tests: tiny seeded graphs and dense algebra.

Dense matrices here are built from the edge lists directly (Eq.
formula_laplacian), independently of both the oracle and the GPU library.
"""
from __future__ import annotations

import numpy as np

from synth import graphs, rng


def tiny_graph(n: int, extra: int, seed: int, integer_weights: bool = False, D: float = 0.0):
    """Connected graph: a random spanning path plus `extra` random edges."""
    perm = np.argsort(rng.uniform(seed, 11, n))
    edges = set()
    for i in range(n - 1):
        a, b = int(perm[i]), int(perm[i + 1])
        edges.add((min(a, b), max(a, b)))
    draws = rng.raw64(seed, 12, 0, 8 * extra + 16)
    k = 0
    while len(edges) < n - 1 + extra and k + 1 < draws.shape[0]:
        a, b = int(draws[k] % np.uint64(n)), int(draws[k + 1] % np.uint64(n))
        k += 2
        if a != b:
            edges.add((min(a, b), max(a, b)))
    e = np.array(sorted(edges), dtype=np.int64)
    if integer_weights:
        w = 1.0 + (rng.raw64(seed, 13, 0, e.shape[0]) % np.uint64(3)).astype(np.float64)
    else:
        w = 0.5 + 4.5 * rng.uniform(seed, 13, e.shape[0])
    rowptr, col, val = graphs.csr_from_edges(n, e[:, 0], e[:, 1], w, D)
    return graphs.Graph(f"tiny{n}_{seed}", n, rowptr, col, val)


def dense_from_csr(g) -> np.ndarray:
    A = np.zeros((g.n, g.n))
    for p in range(g.n):
        for j in range(g.rowptr[p], g.rowptr[p + 1]):
            A[p, g.col[j]] = g.val[j]
    return A


def dense_lap(n, eu, ev, ew, mask=None) -> np.ndarray:
    L = np.zeros((n, n))
    for e in range(len(eu)):
        if mask is not None and not mask[e]:
            continue
        a, b, w = int(eu[e]), int(ev[e]), float(ew[e])
        L[a, a] += w
        L[b, b] += w
        L[a, b] -= w
        L[b, a] -= w
    return L


def tree_path(n, eu, ev, in_tree, p, q):
    """Edge ids on the tree path p -> q (BFS in plain Python)."""
    adj = {v: [] for v in range(n)}
    for e in np.flatnonzero(in_tree):
        adj[int(eu[e])].append((int(ev[e]), int(e)))
        adj[int(ev[e])].append((int(eu[e]), int(e)))
    prev = {p: None}
    stack = [p]
    while stack:
        v = stack.pop()
        for c, e in adj[v]:
            if c not in prev:
                prev[c] = (v, e)
                stack.append(c)
    path = []
    v = q
    while prev[v] is not None:
        v, e = prev[v]
        path.append(e)
    return path


def gen_eigs(LG, LS, ground=0):
    """Generalized eigenvalues of L_G u = lambda L_S u on the complement of 1
    (ground one vertex: both reduced matrices are SPD for connected S)."""
    import scipy.linalg
    keep = [i for i in range(LG.shape[0]) if i != ground]
    return scipy.linalg.eigh(LG[np.ix_(keep, keep)], LS[np.ix_(keep, keep)], eigvals_only=True)
