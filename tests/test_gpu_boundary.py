"""The boundary calls beyond the five core ones, through the C ABI, against
the oracle: the caller's spanning tree (grass_tree_from_edges), the host
export of a sparsifier (grass_sparsifier_edges), the similarity check of
Sec. IV-D step 6 (grass_filter_similar and grass_densify with the check on),
and the hair-comb experiment of Sec. V-C built on a caller's tree.

Tolerances: edge sets and ids bit-exact (the same heats go to both sides
where a filter decision is compared); FP64 heats 1e-10 of heat_max.
"""
import numpy as np
import pytest

import oracle
from synth import graphs, rng
from tests.gpu_util import dev, gpu_graph, host, tree_mask

pytestmark = pytest.mark.gpu

HEAT_TOL = 1e-10


def _comb_ids(og, nx, ny):
    u, v = graphs.hair_comb_edges(nx, ny)
    key = og.eu.astype(np.int64) * og.n + og.ev
    ids = np.searchsorted(key, u * og.n + v)
    assert np.array_equal(key[ids], u * og.n + v)
    return ids.astype(np.int64)


def _user_tree(gpu, ctx, g, ids, ground=0):
    return gpu.grass_tree_from_edges(ctx, dev(g.rowptr), dev(g.col), dev(g.val), dev(ids), ground)


# ---------------------------------------------------------------- caller's tree

def test_tree_from_edges_comb_heats_and_solve_match_oracle(gpu):
    import torch
    g = graphs.grid2d_uniform(41, 29, seed=81)
    og = oracle.from_graph(g)
    ids = _comb_ids(og, 41, 29)
    in_tree = np.zeros(og.m, np.uint8)
    in_tree[ids] = 1
    ot = oracle.orient(og, in_tree, 0)
    perm = ids[np.argsort(rng.uniform(81, 5, ids.shape[0]))]       # any order
    ctx = gpu.grass_ctx_create()
    tree = None
    try:
        tree = _user_tree(gpu, ctx, g, perm)
        assert np.array_equal(tree_mask(ctx, tree, og.m), in_tree)
        # tree solve with and without D
        B = rng.gaussian_block(81, 6, g.n, 8)
        for with_D in (0, 1):
            ref = oracle.tree_solve(og, ot, B - B.mean(axis=0) if not with_D else B,
                                    og.D if with_D else None)
            Bd = dev(B - B.mean(axis=0) if not with_D else B)
            X = torch.empty_like(Bd)
            gpu.grass_tree_solve(ctx, tree, with_D, 8, gpu.GRASS_FP64, Bd, X)
            x = host(X)
            if not with_D:      # grounded at vertex 0: compare up to the constant
                x = x - x.mean(axis=0)
                ref = ref - ref.mean(axis=0)
            assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()
        # the embedding's heats on the comb
        h0 = rng.gaussian_block(81, rng.STREAM_H0, g.n, 4)
        H = oracle.embed(og, ot, None, h0, 2)
        hv_ref, off_ref = oracle.heat(og, in_tree, H)
        S = gpu.grass_sparsifier_create(ctx, tree)
        try:
            heat = torch.empty(off_ref.shape[0], dtype=torch.float64, device="cuda")
            gpu.grass_embed(ctx, S, dev(h0), 4, 2, gpu.GRASS_FP64, 1e-12, 100, None, heat)
            hv = host(heat)
            assert np.abs(hv / hv.max() - hv_ref / hv_ref.max()).max() <= HEAT_TOL
        finally:
            gpu.grass_sparsifier_destroy(S)
    finally:
        if tree:
            gpu.grass_tree_destroy(tree)
        gpu.grass_ctx_destroy(ctx)


def test_tree_from_edges_rejects_non_trees(gpu):
    g = graphs.grid2d_uniform(12, 9, seed=82)
    og = oracle.from_graph(g)
    ids = _comb_ids(og, 12, 9)
    ctx = gpu.grass_ctx_create()
    try:
        bad = ids.copy()
        bad[3] = og.m                                    # out of range
        dup = ids.copy()
        dup[5] = dup[6]                                  # repeated id
        # a cycle: drop a tooth edge, add the horizontal edge that closes a
        # cycle with the spine and two teeth (n - 1 distinct ids, not a tree)
        cyc = ids.copy()
        tooth = np.flatnonzero((og.eu[ids] == 3 * 12 + 5) & (og.ev[ids] == 4 * 12 + 5))[0]
        across = np.flatnonzero((og.eu == 2 * 12 + 5) & (og.ev == 2 * 12 + 6))[0]
        cyc[tooth] = across
        for ids_bad in (bad, dup, cyc):
            with pytest.raises(gpu.GrassError) as e:
                _user_tree(gpu, ctx, g, ids_bad)
            assert e.value.status == gpu.GRASS_ERR_INVALID
        # still usable: the valid tree builds
        tree = _user_tree(gpu, ctx, g, ids)
        gpu.grass_tree_destroy(tree)
    finally:
        gpu.grass_ctx_destroy(ctx)


# ---------------------------------------------------------------- sparsifier export

def test_sparsifier_edges_host_export(gpu):
    import torch
    g = graphs.grid3d_loguniform(11, 9, 7, seed=83)
    og = oracle.from_graph(g)
    with gpu_graph(g) as (ctx, tree, _):
        S = gpu.grass_sparsifier_create(ctx, tree)
        try:
            ids, cnt = gpu.grass_sparsifier_edges(S)
            ot_mask = tree_mask(ctx, tree, og.m)
            assert cnt == g.n - 1 and np.array_equal(ids, np.flatnonzero(ot_mask))
            off = np.flatnonzero(ot_mask == 0)
            gpu.grass_sparsifier_add(ctx, S, dev(off[::3].astype(np.int64)))
            ids, cnt = gpu.grass_sparsifier_edges(S)
            mask = torch.empty(og.m, dtype=torch.uint8, device="cuda")
            gpu.grass_sparsifier_mask(ctx, S, mask)
            assert np.array_equal(ids, np.flatnonzero(host(mask)))
            assert cnt == ids.shape[0] == g.n - 1 + off[::3].shape[0]
            part, cnt2 = gpu.grass_sparsifier_edges(S, 10)
            assert cnt2 == cnt and np.array_equal(part, ids[:10])
            none, cnt3 = gpu.grass_sparsifier_edges(S, 0)
            assert cnt3 == cnt and none.shape[0] == 0
        finally:
            gpu.grass_sparsifier_destroy(S)


# ---------------------------------------------------------------- similarity check (step 6)

@pytest.mark.parametrize("cap", [0, 1, 57])
def test_filter_similar_matches_oracle(gpu, cap):
    import torch
    g = graphs.grid2d_uniform(45, 38, seed=84)
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    H = oracle.embed(og, ot, None, rng.gaussian_block(84, 1, g.n, 8), 2)
    hv, off = oracle.heat(og, ot.in_tree, H)
    ties = np.round(hv / hv.max() * 40.0)           # integer heats: many ties
    with gpu_graph(g) as (ctx, tree, _):
        S = gpu.grass_sparsifier_create(ctx, tree)
        try:
            acc = torch.empty(max(1, off.shape[0]), dtype=torch.int64, device="cuda")
            for h, th_args in ((hv, (100.0, 1.0, 6000.0, 2)), (ties, (1.0, 1.0, 100.0, 1))):
                theta = oracle.theta_sigma(th_args[0], th_args[1], th_args[2], th_args[3])
                ref = oracle.similarity_check(og, h, off, theta, cap)
                na, th = gpu.grass_filter_similar(ctx, S, dev(h), gpu.GRASS_FP64, *th_args, cap, acc)
                assert th == theta
                assert np.array_equal(host(acc)[:na], ref)
                # FP32 heats: the same rule on the rounded values
                h32 = h.astype(np.float32)
                na32, _ = gpu.grass_filter_similar(ctx, S, dev(h32), gpu.GRASS_FP32, *th_args, cap,
                                                   acc)
                ref32 = oracle.similarity_check(
                    og, h32.astype(np.float64), off,
                    theta * float(h32.max()) / float(h32.astype(np.float64).max()), cap)
                assert np.array_equal(host(acc)[:na32], ref32)
        finally:
            gpu.grass_sparsifier_destroy(S)


@pytest.mark.parametrize("which", ["grid64", "grid3d"])
def test_densify_with_similarity_check_matches_oracle(gpu, which):
    import torch
    if which == "grid64":
        g, sigma2, r, rounds, cap = graphs.config_small_grid(), 100.0, 8, 1, 0
    else:
        g, sigma2, r, rounds, cap = graphs.grid3d_loguniform(12, 12, 12, seed=2), 20.0, 16, 3, 60
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    h0s = [rng.gaussian_block(9, rng.STREAM_H0 + k, g.n, r) for k in range(rounds)]
    v0s = [rng.normal(9, rng.STREAM_V0 + k, g.n) for k in range(rounds)]
    res = oracle.densify(og, ot, h0s, v0s, sigma2, 2, rounds, 8, cap, 1e-13, 3000,
                         record=True, similarity=True)
    with gpu_graph(g) as (ctx, tree, _):
        gpu.grass_ctx_set_param(ctx, "similarity_check", 1)
        P = gpu.make_params(sigma2, r, 2, rounds, 8, cap, gpu.GRASS_FP64, 1e-13, 3000)
        S, st = gpu.grass_densify(ctx, tree, P, dev(np.concatenate(h0s)), dev(np.concatenate(v0s)))
        try:
            mask = torch.empty(og.m, dtype=torch.uint8, device="cuda")
            gpu.grass_sparsifier_mask(ctx, S, mask)
            got = host(mask)
            d = st.as_dict()
            assert d["rounds"] == res.rounds and d["added_round"] == res.added
            assert np.array_equal(got, res.in_s)
            # every round's additions form a matching (no shared endpoint)
            add = np.flatnonzero((got == 1) & (ot.in_tree == 0))
            if rounds == 1:
                ends = np.concatenate([og.eu[add], og.ev[add]])
                assert np.unique(ends).shape[0] == ends.shape[0]
        finally:
            gpu.grass_sparsifier_destroy(S)


# ---------------------------------------------------------------- hair comb (Sec. V-C)

def test_hair_comb_200(gpu):
    """The 200 x 200 unit mesh with the hair-comb spanning tree: the tree's
    lambda_max estimate (eight power steps, Sec. V-B) is about 64,000 as the
    paper states; one random vector and one power step (t = 1) give heats
    equal to the oracle's and the same 400 most critical edges."""
    import torch
    k = 200
    g = graphs.grid((k, k), None, 0.0)
    og = oracle.from_graph(g)
    ids = _comb_ids(og, k, k)
    in_tree = np.zeros(og.m, np.uint8)
    in_tree[ids] = 1
    ot = oracle.orient(og, in_tree, 0)
    h0 = rng.gaussian_block(3, rng.STREAM_H0, g.n, 1)
    H = oracle.embed(og, ot, None, h0, 1)
    hv_ref, off = oracle.heat(og, in_tree, H)
    top_ref = oracle.filter_edges(hv_ref, off, 0.0, 400)
    v0 = rng.normal(3, rng.STREAM_V0, g.n)
    ctx = gpu.grass_ctx_create()
    tree = None
    try:
        tree = _user_tree(gpu, ctx, g, ids)
        S = gpu.grass_sparsifier_create(ctx, tree)
        try:
            lmax = gpu.grass_lambda_max(ctx, S, dev(v0), 8, gpu.GRASS_FP64, 1e-12, 100)
            assert 0.85 * 64000.0 <= lmax <= 1.05 * 64000.0
            heat = torch.empty(off.shape[0], dtype=torch.float64, device="cuda")
            gpu.grass_embed(ctx, S, dev(h0), 1, 1, gpu.GRASS_FP64, 1e-12, 100, None, heat)
            hv = host(heat)
            assert np.abs(hv / hv.max() - hv_ref / hv_ref.max()).max() <= HEAT_TOL
            acc = torch.empty(off.shape[0], dtype=torch.int64, device="cuda")
            # theta -> 0: every edge passes the threshold, the cap keeps the top 400
            na, _ = gpu.grass_filter(ctx, S, heat, gpu.GRASS_FP64, 1e-30, 1.0, 1.0, 1, 400, acc)
            assert na == 400 and np.array_equal(host(acc)[:na], top_ref)
        finally:
            gpu.grass_sparsifier_destroy(S)
    finally:
        if tree:
            gpu.grass_tree_destroy(tree)
        gpu.grass_ctx_destroy(ctx)


# ---------------------------------------------------------------- grid share

@pytest.mark.parametrize("grid_sms", [8, 37])
def test_grid_sms_share_keeps_results(gpu, grid_sms):
    """Cooperative kernels on a share of the SMs (the serving knob): the tree
    solve matches the oracle, the fused PCG reaches its tolerance (checked
    with the oracle's product), and repeated runs under the same share are
    bit-identical."""
    import torch
    g = graphs.grid3d_loguniform(22, 19, 17, seed=90)
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og, 0)
    B = rng.gaussian_block(90, 6, g.n, 8)
    ref = oracle.tree_solve(og, ot, B, og.D)
    b = rng.normal(90, rng.STREAM_RHS, g.n)
    with gpu_graph(g) as (ctx, tree, (rp, col, val)):
        gpu.grass_ctx_set_param(ctx, "grid_sms", grid_sms)
        X = torch.empty(g.n, 8, dtype=torch.float64, device="cuda")
        gpu.grass_tree_solve(ctx, tree, 1, 8, gpu.GRASS_FP64, dev(B), X)
        assert np.abs(host(X) - ref).max() <= 1e-10 * np.abs(ref).max()
        S = gpu.grass_sparsifier_create(ctx, tree)
        try:
            xs = []
            for _ in range(2):
                x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
                st, ps = gpu.grass_pcg_solve(ctx, S, dev(b), x, 1e-8, 4000, gpu.GRASS_FP32, 1e-2,
                                             1e-2, 1)
                assert st == 0 and ps.rel_resid_fp64 <= 1e-8
                xs.append(host(x))
            assert np.array_equal(xs[0], xs[1])
            A = oracle.lap_apply(og, xs[0]) + og.D * xs[0]
            assert np.linalg.norm(b - A) <= 1.01e-8 * np.linalg.norm(b)
        finally:
            gpu.grass_sparsifier_destroy(S)
