"""The scan form of the grounded tree solve (Euler tour + two FP64 prefix
sums; one column, no D) against the oracle's leaf-first elimination and
against the library's own elimination-round solve.

Trees: 2D/3D grids, a ring (its spanning tree is a path: depth n), a
power-law graph (hubs of high degree), a power grid, tiny random graphs,
and a forest of several graphs.
"""
import numpy as np
import pytest

import oracle
from synth import graphs, rng
from tests.gpu_util import dev, gpu_graph, host
from tests.helpers import tiny_graph

pytestmark = pytest.mark.gpu


def _cases():
    return [graphs.grid2d_uniform(40, 30, seed=3), graphs.grid3d_loguniform(12, 11, 10, seed=4),
            graphs.ring_chords(3000, seed=5, chord_frac=0.0), graphs.chung_lu(6000, seed=6),
            graphs.power_grid(50, 7), tiny_graph(9, 4, seed=8), tiny_graph(2, 0, seed=9)]


def _solve(gpu, ctx, tree, b, prec, euler):
    import torch
    gpu.grass_ctx_set_param(ctx, "euler_solve", 1 if euler else 0)
    B = dev(b) if prec == gpu.GRASS_FP64 else dev(b).float()
    X = torch.empty_like(B)
    gpu.grass_tree_solve(ctx, tree, 0, 1, prec, B, X)
    return host(X).astype(np.float64)


@pytest.mark.parametrize("gi", range(7))
def test_scan_solve_matches_oracle_and_elimination(gpu, gi):
    g = _cases()[gi]
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og, 0)
    b = rng.normal(50 + gi, 7, g.n)
    b -= b.mean()
    ref = oracle.tree_solve(og, ot, b)
    scale = np.abs(ref).max()
    with gpu_graph(g) as (ctx, tree, _):
        x_eu = _solve(gpu, ctx, tree, b, gpu.GRASS_FP64, True)
        x_el = _solve(gpu, ctx, tree, b, gpu.GRASS_FP64, False)
        x32 = _solve(gpu, ctx, tree, b, gpu.GRASS_FP32, True)
    assert x_eu[0] == 0.0
    assert np.abs(x_eu - ref).max() <= 1e-10 * scale
    assert np.abs(x_eu - x_el).max() <= 1e-10 * scale
    assert np.abs(x32 - ref).max() <= 1e-5 * scale


def test_scan_solve_on_a_forest(gpu):
    import torch
    gs = _cases()[:5]
    u, off = graphs.batch_union(gs)
    parts = []
    for k, g in enumerate(gs):
        bk = rng.normal(60 + k, 7, g.n)
        parts.append(bk - bk.mean())
    b = np.concatenate(parts)
    ctx = gpu.grass_ctx_create()
    try:
        rp, col, val = dev(u.rowptr), dev(u.col), dev(u.val)
        tree = gpu.grass_build_forest(ctx, rp, col, val, off)
        try:
            x = _solve(gpu, ctx, tree, b, gpu.GRASS_FP64, True)
        finally:
            gpu.grass_tree_destroy(tree)
    finally:
        gpu.grass_ctx_destroy(ctx)
    for k, g in enumerate(gs):
        og = oracle.from_graph(g)
        ot = oracle.build_tree(og, 0)
        ref = oracle.tree_solve(og, ot, parts[k])
        xk = x[off[k]:off[k + 1]]
        assert xk[0] == 0.0
        assert np.abs(xk - ref).max() <= 1e-10 * np.abs(ref).max(), k


def test_lambda_max_through_inner_cg_with_scan_solves(gpu):
    """lambda_max of a sparsifier with off-tree edges: its power steps run the
    fused inner CG, whose preconditioner is now the scan-form solve."""
    import torch
    g = graphs.grid2d_uniform(45, 40, seed=12)
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og, 0)
    in_s = ot.in_tree.copy()
    off = np.flatnonzero(in_s == 0)
    in_s[off[::7]] = 1
    v0 = rng.normal(13, rng.STREAM_V0, g.n)
    ref = oracle.lambda_max_est(og, ot, in_s, v0, 6, 1e-13, 3000)
    with gpu_graph(g) as (ctx, tree, _):
        S = gpu.grass_sparsifier_create(ctx, tree)
        try:
            gpu.grass_sparsifier_add(ctx, S, dev(off[::7].astype(np.int64)))
            vals = {}
            for eu in (1, 0):
                gpu.grass_ctx_set_param(ctx, "euler_solve", eu)
                vals[eu] = gpu.grass_lambda_max(ctx, S, dev(v0), 6, gpu.GRASS_FP64, 1e-13, 3000)
        finally:
            gpu.grass_sparsifier_destroy(S)
    assert abs(vals[1] - ref) <= 1e-9 * ref
    assert abs(vals[1] - vals[0]) <= 1e-9 * ref
