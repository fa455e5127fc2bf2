"""The low-stretch spanning tree (grass_build_lsst) and the per-edge stretch
(grass_tree_stretch) through the C ABI, against the oracle.

The tree is a function of (graph, seed): bit-exact against the oracle's on
meshes, weighted 3D grids, random graphs, a power grid, a power-law graph,
a ring with chords and the degenerate cases.  Stretch: FP64 per edge within
1e-9 relative (sums of path resistances taken in another order; the
subtraction R(u) + R(v) - 2 R(lca) loses about depth x eps relative to R),
total within 1e-9.  At a size the oracle cannot walk (60^3), the tree is
checked by what holds at any size: n - 1 edges with no cycle (re-validated by
grass_tree_from_edges), the class-forest property against scipy's connected
components, and the stretch of sampled edges by walking the tree on the CPU.
"""
import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle
from synth import graphs, rng
from tests.gpu_util import dev, host, tree_mask

pytestmark = pytest.mark.gpu

ST_TOL = 1e-9


def _lsst(gpu, ctx, g, seed, ground=0):
    return gpu.grass_build_lsst(ctx, dev(g.rowptr), dev(g.col), dev(g.val), seed, ground)


def _graph(u, v, w, n, D=0.0):
    rowptr, col, val = graphs.csr_from_edges(n, np.asarray(u), np.asarray(v),
                                             np.asarray(w, dtype=np.float64), D)
    return graphs.Graph("edges", n, rowptr, col, val)


def _random_graph(n, extra, seed):
    r = np.random.default_rng(seed)
    perm = r.permutation(n)
    pairs = {(int(min(perm[i], perm[j])), int(max(perm[i], perm[j])))
             for i, j in ((i, int(r.integers(0, i))) for i in range(1, n))}
    while len(pairs) < n - 1 + extra:
        a, b = r.integers(0, n, 2)
        if a != b:
            pairs.add((int(min(a, b)), int(max(a, b))))
    pairs = sorted(pairs)
    u = [p[0] for p in pairs]
    v = [p[1] for p in pairs]
    # a few weights repeated so that equal-weight ties are decided by id
    w = 2.0 ** r.uniform(-5, 5, len(pairs))
    w[r.integers(0, len(pairs), len(pairs) // 4)] = 1.0
    return _graph(u, v, w, n, 1e-3)


CASES = {
    "unit_mesh_48": lambda: graphs.grid((48, 48)),
    "unit_mesh_odd_37x23": lambda: graphs.grid((37, 23)),
    "loguniform_3d_12": lambda: graphs.grid3d_loguniform(12, 12, 12, 5),
    "uniform_mesh_40": lambda: graphs.grid2d_uniform(40, 40, 3),
    "power_grid_40": lambda: graphs.power_grid(40, 6),
    "ring_chords_3000": lambda: graphs.ring_chords(3000, 4),
    "chung_lu_4000": lambda: graphs.chung_lu(4000, 9),
    "random_500": lambda: _random_graph(500, 900, 12),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("seed", [1, 0xDEADBEEFCAFE])
def test_lsst_bit_exact(gpu, name, seed):
    g = CASES[name]()
    og = oracle.from_graph(g)
    want = oracle.low_stretch_tree(og, seed=seed)
    ctx = gpu.grass_ctx_create()
    tree = None
    try:
        tree, st = _lsst(gpu, ctx, g, seed)
        got = tree_mask(ctx, tree, og.m)
        assert np.array_equal(got, want), (name, int((got != want).sum()))
        assert st["classes"] == int(oracle.lsst_classes(og.ew).max()) + 1
        assert st["levels"] >= 1 and st["rounds"] >= st["levels"]
    finally:
        if tree:
            gpu.grass_tree_destroy(tree)
        gpu.grass_ctx_destroy(ctx)


def test_lsst_degenerate_cases(gpu):
    cases = [
        _graph([0], [1], [2.5], 2),                                   # one edge
        _graph(np.arange(9), np.arange(1, 10), np.ones(9), 10),       # a path
        _graph(np.zeros(7, int), np.arange(1, 8), 2.0 ** np.arange(7), 8),   # a star
        _graph([0, 0, 1, 2], [1, 2, 2, 3], [1.0, 1.0, 1.0, 1.0], 4),  # all weights equal
        _graph([0, 1, 0], [1, 2, 2], [1e-300, 1e300, 1.0], 3),        # extreme binades
    ]
    for g in cases:
        og = oracle.from_graph(g)
        want = oracle.low_stretch_tree(og, seed=7)
        ctx = gpu.grass_ctx_create()
        tree = None
        try:
            tree, _ = _lsst(gpu, ctx, g, 7)
            assert np.array_equal(tree_mask(ctx, tree, og.m), want)
        finally:
            if tree:
                gpu.grass_tree_destroy(tree)
            gpu.grass_ctx_destroy(ctx)


def test_lsst_disconnected_is_an_error(gpu):
    g = _graph([0, 2], [1, 3], [1.0, 1.0], 4)
    ctx = gpu.grass_ctx_create()
    try:
        with pytest.raises(gpu.GrassError) as ei:
            _lsst(gpu, ctx, g, 1)
        assert ei.value.status == 3      # GRASS_ERR_DISCONNECTED
    finally:
        gpu.grass_ctx_destroy(ctx)


@pytest.mark.parametrize("kind", ["mst", "lsst"])
@pytest.mark.parametrize("name", ["unit_mesh_48", "loguniform_3d_12", "power_grid_40",
                                  "chung_lu_4000"])
def test_stretch_matches_oracle(gpu, kind, name):
    import torch
    g = CASES[name]()
    og = oracle.from_graph(g)
    ctx = gpu.grass_ctx_create()
    tree = None
    try:
        if kind == "mst":
            tree = gpu.grass_build_tree(ctx, dev(g.rowptr), dev(g.col), dev(g.val), 0)
        else:
            tree, _ = _lsst(gpu, ctx, g, 3)
        in_tree = tree_mask(ctx, tree, og.m)
        want_tot, want = oracle.total_stretch(og, in_tree)
        st = torch.empty(og.m, dtype=torch.float64, device="cuda")
        tot = gpu.grass_tree_stretch(ctx, tree, st)
        got = host(st)
        assert np.all(np.abs(got - want) <= ST_TOL * np.maximum(1.0, want))
        assert abs(tot - want_tot) <= ST_TOL * want_tot
        assert abs(gpu.grass_tree_stretch(ctx, tree) - tot) == 0.0   # deterministic
    finally:
        if tree:
            gpu.grass_tree_destroy(tree)
        gpu.grass_ctx_destroy(ctx)


def test_lsst_lowers_stretch_on_unit_mesh(gpu):
    g = graphs.grid((128, 128))
    ctx = gpu.grass_ctx_create()
    t1 = t2 = None
    try:
        t1 = gpu.grass_build_tree(ctx, dev(g.rowptr), dev(g.col), dev(g.val), 0)
        t2, _ = _lsst(gpu, ctx, g, 1)
        s_mst = gpu.grass_tree_stretch(ctx, t1)
        s_lsst = gpu.grass_tree_stretch(ctx, t2)
        assert s_lsst < 0.25 * s_mst
    finally:
        for t in (t1, t2):
            if t:
                gpu.grass_tree_destroy(t)
        gpu.grass_ctx_destroy(ctx)


def test_lsst_full_size_properties(gpu):
    """60^3 log-uniform grid (216,000 vertices): the tree re-validates as a
    spanning tree, its class-<=c edges span every component of G_{<=c}, and
    sampled stretches agree with tree walks on the CPU."""
    import torch
    g = graphs.grid3d_loguniform(60, 60, 60, 2)
    og = oracle.from_graph(g)
    n = og.n
    ctx = gpu.grass_ctx_create()
    t1 = t2 = None
    try:
        t1, _ = _lsst(gpu, ctx, g, 1)
        in_tree = tree_mask(ctx, t1, og.m)
        ids = np.flatnonzero(in_tree).astype(np.int64)
        assert ids.shape[0] == n - 1
        t2 = gpu.grass_tree_from_edges(ctx, dev(g.rowptr), dev(g.col), dev(g.val), dev(ids), 0)
        cls = oracle.lsst_classes(og.ew)
        for c in range(int(cls.max()) + 1):
            sub = np.flatnonzero(cls <= c)
            a = coo_matrix((np.ones(sub.shape[0]), (og.eu[sub], og.ev[sub])), shape=(n, n))
            comps = connected_components(a, directed=False)[0]
            assert int(((in_tree != 0) & (cls <= c)).sum()) == n - comps, c
        st = torch.empty(og.m, dtype=torch.float64, device="cuda")
        gpu.grass_tree_stretch(ctx, t1, st)
        got = host(st)
        tr = oracle.orient(og, in_tree, 0)
        depth = np.zeros(n, np.int64)
        dist = np.zeros(n)
        for v in tr.order[1:]:
            depth[v] = depth[tr.parent[v]] + 1
            dist[v] = dist[tr.parent[v]] + 1.0 / tr.pw[v]
        sample = (rng.uniform(60, 1, 2000) * og.m).astype(np.int64)
        for e in sample:
            a, b = int(og.eu[e]), int(og.ev[e])
            p, q = a, b
            while depth[p] > depth[q]:
                p = tr.parent[p]
            while depth[q] > depth[p]:
                q = tr.parent[q]
            while p != q:
                p, q = tr.parent[p], tr.parent[q]
            want = og.ew[e] * (dist[a] + dist[b] - 2.0 * dist[p])
            assert abs(got[e] - want) <= ST_TOL * max(1.0, want)
    finally:
        for t in (t1, t2):
            if t:
                gpu.grass_tree_destroy(t)
        gpu.grass_ctx_destroy(ctx)
