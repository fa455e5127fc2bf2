"""The batched form: several graphs as one block-diagonal matrix.

* the spanning forest is bit-exact against Kruskal on every graph, and the
  forest solve matches the oracle's tree solve of each graph (grounded at
  its first vertex, and with D);
* one densification round over the batch gives, per graph, the oracle's
  lambda estimates and accepted edge set (edges within 1e-9 of the
  threshold excepted);
* the batched PCG meets the tolerance on every graph (FP64 residual on the
  host) for both vector precisions;
* a graph's results are bit-identical whether it is solved inside the batch
  or alone, and with or without the CUDA-graph replay;
* the autotuner keeps the solve's results bit-identical;
* a batch with an edge between graphs, or a disconnected graph, is refused.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from synth import graphs, rng
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu

R, T, SIGMA2 = 8, 2, 100.0


def _batch():
    return [graphs.grid2d_uniform(20, 15, seed=11), graphs.ring_chords(700, seed=12),
            graphs.power_grid(30, 13), graphs.grid2d_uniform(33, 17, seed=14),
            graphs.ring_chords(90, seed=15), graphs.grid2d_uniform(70, 64, seed=16)]


def _inputs(gs, off, seed=21):
    h0 = np.concatenate([rng.gaussian_block(seed + k, rng.STREAM_H0, g.n, R) for k, g in enumerate(gs)])
    v0 = np.concatenate([rng.normal(seed + k, rng.STREAM_V0, g.n) for k, g in enumerate(gs)])
    b = np.concatenate([rng.normal(seed + k, rng.STREAM_RHS, g.n) for k, g in enumerate(gs)])
    return h0, v0, b


class Forest:
    def __init__(self, gpu, gs, stream=None):
        import torch
        self.gpu, self.gs = gpu, gs
        self.u, self.off = graphs.batch_union(gs)
        self.ctx = gpu.grass_ctx_create(stream)
        self.rp, self.col, self.val = dev(self.u.rowptr), dev(self.u.col), dev(self.u.val)
        self.tree = gpu.grass_build_forest(self.ctx, self.rp, self.col, self.val, self.off)
        self.voff, self.eoff = gpu.grass_tree_segments(self.tree)

    def close(self):
        self.gpu.grass_tree_destroy(self.tree)
        self.gpu.grass_ctx_destroy(self.ctx)


@pytest.fixture
def forest(gpu):
    f = Forest(gpu, _batch())
    yield f
    f.close()


def test_forest_is_kruskal_per_graph_and_solves_match(gpu, forest):
    import torch
    gs, off = forest.gs, forest.off
    assert forest.voff == off
    in_tree = torch.empty(int(forest.eoff[-1]), dtype=torch.uint8, device="cuda")
    gpu.grass_tree_edges(forest.ctx, forest.tree, in_tree)
    it = host(in_tree)
    # right-hand sides summing to zero on every graph (the range of L_T)
    Bs = [rng.gaussian_block(31 + k, 6, g.n, 4) for k, g in enumerate(gs)]
    B = np.concatenate([Bk - Bk.mean(axis=0) for Bk in Bs])
    Bd = dev(B)
    X0, X1 = torch.empty_like(Bd), torch.empty_like(Bd)
    gpu.grass_tree_solve(forest.ctx, forest.tree, 0, 4, gpu.GRASS_FP64, Bd, X0)
    gpu.grass_tree_solve(forest.ctx, forest.tree, 1, 4, gpu.GRASS_FP64, Bd, X1)
    x0, x1 = host(X0), host(X1)
    for k, g in enumerate(gs):
        og = oracle.from_graph(g)
        ot = oracle.build_tree(og, 0)
        assert np.array_equal(it[forest.eoff[k]:forest.eoff[k + 1]], ot.in_tree), k
        Bk = B[off[k]:off[k + 1]]
        ref0 = oracle.tree_solve(og, ot, Bk)
        ref1 = oracle.tree_solve(og, ot, Bk, og.D)
        assert np.all(x0[off[k]] == 0.0)
        assert np.abs(x0[off[k]:off[k + 1]] - ref0).max() <= 1e-10 * np.abs(ref0).max(), k
        assert np.abs(x1[off[k]:off[k + 1]] - ref1).max() <= 1e-10 * np.abs(ref1).max(), k


def test_densify_batch_matches_oracle_per_graph(gpu, forest):
    import torch
    gs, off = forest.gs, forest.off
    h0, v0, b = _inputs(gs, off)
    P = gpu.make_params(SIGMA2, R, T, 1, 8, 0, gpu.GRASS_FP64, 1e-12, 2000)
    S, st, rows = gpu.grass_densify_batch(forest.ctx, forest.tree, P, dev(h0), dev(v0), len(gs))
    try:
        in_s = torch.empty(int(forest.eoff[-1]), dtype=torch.uint8, device="cuda")
        gpu.grass_sparsifier_mask(forest.ctx, S, in_s)
        mask = host(in_s)
    finally:
        gpu.grass_sparsifier_destroy(S)
    added = 0
    for k, g in enumerate(gs):
        og = oracle.from_graph(g)
        ot = oracle.build_tree(og, 0)
        res = oracle.densify(og, ot, [h0[off[k]:off[k + 1]]], [v0[off[k]:off[k + 1]]], SIGMA2, T, 1,
                             8, 0, 1e-12, 2000)
        lmin, lmax, theta, hmax, nadd, nemb = rows[k]
        assert abs(lmin - res.lmin[0]) <= 1e-14 * res.lmin[0], k
        assert abs(lmax - res.lmax[0]) <= 1e-9 * res.lmax[0], k
        mk = mask[forest.eoff[k]:forest.eoff[k + 1]]
        if res.stopped_similar:
            assert np.isinf(theta) and nadd == 0 and np.array_equal(mk, ot.in_tree), k
            continue
        diff = np.flatnonzero(mk != res.in_s)
        if diff.size:
            # only edges whose heat lies within 1e-9 of the threshold may differ
            H = oracle.embed(og, ot, None, h0[off[k]:off[k + 1]], T)
            hv, offe = oracle.heat(og, ot.in_tree, H)
            thr = res.theta[0] * hv.max()
            pos = np.searchsorted(offe, diff)
            assert np.all(np.abs(hv[pos] - thr) <= 1e-9 * thr), (k, diff)
        assert int(nadd) == int(mk.sum() - ot.in_tree.sum()), k
        added += int(nadd)
    assert st.added == added


def _rel_resid(g, x, b):
    A = sp.csr_matrix((g.val, g.col, g.rowptr), shape=(g.n, g.n))
    return np.linalg.norm(b - A @ x) / np.linalg.norm(b)


def _solve(gpu, fr, h0, v0, b, prec, inner, tol=1e-6):
    import torch
    P = gpu.make_params(SIGMA2, R, T, 1, 8, 0, gpu.GRASS_FP32, 1e-2, 30)
    S, st, rows = gpu.grass_densify_batch(fr.ctx, fr.tree, P, dev(h0), dev(v0), len(fr.gs))
    try:
        x = torch.zeros(fr.u.n, dtype=torch.float64, device="cuda")
        s, ps, its, res = gpu.grass_pcg_solve_batch(fr.ctx, S, dev(b), x, tol, 3000, prec, inner,
                                                     len(fr.gs))
    finally:
        gpu.grass_sparsifier_destroy(S)
    return s, ps, its, res, host(x), rows


@pytest.mark.parametrize("prec,inner,tol", [(0, 0, 1e-8), (0, 3, 1e-8), (1, 1, 1e-3), (1, 0, 1e-3),
                                            (1, 1, 1e-7)])
def test_pcg_batch_meets_tolerance_per_graph(gpu, forest, prec, inner, tol):
    gs, off = forest.gs, forest.off
    h0, v0, b = _inputs(gs, off)
    s, ps, its, res, x, _ = _solve(gpu, forest, h0, v0, b, prec, inner, tol)
    assert s == 0, (ps.rel_resid_fp64, its)
    for k, g in enumerate(gs):
        rel = _rel_resid(g, x[off[k]:off[k + 1]], b[off[k]:off[k + 1]])
        assert rel <= tol, (k, rel)
        assert abs(rel - res[k]) <= 1e-6 * tol + 1e-12
        assert 1 <= its[k] <= ps.iters


def test_graph_results_do_not_depend_on_the_batch(gpu):
    import torch
    gs = _batch()
    full = Forest(gpu, gs)
    alone = Forest(gpu, [gs[3]])
    stream = torch.cuda.Stream()
    captured = Forest(gpu, gs, stream)
    try:
        h0, v0, b = _inputs(gs, full.off)
        o = full.off
        out_full = _solve(gpu, full, h0, v0, b, 1, 1, 1e-5)
        sl = slice(o[3], o[4])
        out_alone = _solve(gpu, alone, h0[sl], v0[sl], b[sl], 1, 1, 1e-5)
        with torch.cuda.stream(stream):
            out_cap = _solve(gpu, captured, h0, v0, b, 1, 1, 1e-5)
        stream.synchronize()
        assert np.array_equal(out_full[4][sl], out_alone[4])
        assert out_full[2][3] == out_alone[2][0]
        # per-graph lambda_min, lambda_max, theta, edges added, edges embedded
        # (heat_max carries the batch-wide power-of-two scale of the heats)
        keep = [0, 1, 2, 4, 5]
        assert [out_full[5][3][i] for i in keep] == [out_alone[5][0][i] for i in keep]
        assert np.array_equal(out_full[4], out_cap[4])
        assert out_full[2] == out_cap[2]
    finally:
        full.close()
        alone.close()
        captured.close()


def test_autotune_keeps_results(gpu, forest):
    import torch
    B = dev(rng.gaussian_block(41, 6, forest.u.n, 8)).float()
    X0, X1 = torch.empty_like(B), torch.empty_like(B)
    gpu.grass_tree_solve(forest.ctx, forest.tree, 0, 8, gpu.GRASS_FP32, B, X0)
    best, ms = gpu.grass_autotune(forest.ctx, forest.tree, 8, gpu.GRASS_FP32)
    assert best[0] in (256, 512, 1024) and best[1] in (1, 2, 4) and ms > 0
    gpu.grass_tree_solve(forest.ctx, forest.tree, 0, 8, gpu.GRASS_FP32, B, X1)
    assert torch.equal(X0, X1)


def test_bad_batches_are_refused(gpu):
    import torch
    gs = [graphs.grid2d_uniform(6, 5, seed=1), graphs.grid2d_uniform(5, 4, seed=2)]
    u, off = graphs.batch_union(gs)
    ctx = gpu.grass_ctx_create()
    try:
        rp, col, val = dev(u.rowptr), dev(u.col), dev(u.val)
        # offsets that cut graph 0 in two: its edges then join two "graphs"
        with pytest.raises(gpu.GrassError) as e:
            gpu.grass_build_forest(ctx, rp, col, val, [0, 10, u.n])
        assert e.value.status == gpu.GRASS_ERR_INVALID
        # a graph that is itself two components (graph 0 and 1 declared as one)
        with pytest.raises(gpu.GrassError) as e:
            gpu.grass_build_forest(ctx, rp, col, val, [0, u.n])
        assert e.value.status == gpu.GRASS_ERR_DISCONNECTED
        tree = gpu.grass_build_forest(ctx, rp, col, val, off)
        try:
            S = gpu.grass_sparsifier_create(ctx, tree)
            try:
                with pytest.raises(gpu.GrassError) as e:
                    gpu.grass_lambda_min(ctx, S)
                assert e.value.status == gpu.GRASS_ERR_INVALID
            finally:
                gpu.grass_sparsifier_destroy(S)
        finally:
            gpu.grass_tree_destroy(tree)
    finally:
        gpu.grass_ctx_destroy(ctx)
