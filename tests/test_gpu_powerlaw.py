"""The power-law workload (Chung-Lu graphs, unit weights, largest component;
r = 24, t = 3, sigma^2 = 500, FP32 embedding at the benchmark's scale)
against the FP64 oracle, and the FP32 condition-number rule on a larger 3D
grid than the dense eigensolve allows.

* FP64 heats of every off-tree edge agree with the oracle to 1e-10 of
  heat_max on a 1e5-node Chung-Lu graph (hubs of a few hundred neighbours:
  the row kernels' long rows); with unit weights every spanning-tree
  decision is a tie that the edge id breaks, and the tree is bit-exact;
* one densification round (FP64) keeps the oracle's edge set, except edges
  within 1e-9 of a decision (threshold or cap boundary);
* FP32 embeddings give a sparsifier whose condition number (extreme
  generalized eigenvalues by sparse Lanczos, scipy ARPACK) is <= sigma^2
  when the FP64 oracle's is, else within 5 % of the oracle's.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from synth import graphs, rng
from tests.gpu_util import dev, gpu_graph, host, tree_mask
from tests.test_gpu_parity import _near_decision

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pl():
    g = graphs.chung_lu(100_000, seed=31)
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    return g, og, ot


def test_powerlaw_tree_and_heat_match_oracle(gpu, pl):
    import torch
    g, og, ot = pl
    r, t = 24, 3
    deg = np.diff(g.rowptr) - 1
    assert deg.max() >= 200                     # hub rows are exercised
    h0 = rng.gaussian_block(31, rng.STREAM_H0, g.n, r)
    H = oracle.embed(og, ot, None, h0, t)
    ref, off = oracle.heat(og, ot.in_tree, H)
    with gpu_graph(g) as (ctx, tree, _):
        assert np.array_equal(tree_mask(ctx, tree, og.m), ot.in_tree)
        S = gpu.grass_sparsifier_create(ctx, tree)
        try:
            heat = torch.empty(off.shape[0], dtype=torch.float64, device="cuda")
            gpu.grass_embed(ctx, S, dev(h0), r, t, gpu.GRASS_FP64, 1e-10, 100, None, heat)
            hv = host(heat)
            assert np.abs(hv / hv.max() - ref / ref.max()).max() <= 1e-10
            heat32 = torch.empty(off.shape[0], dtype=torch.float32, device="cuda")
            gpu.grass_embed(ctx, S, dev(h0), r, t, gpu.GRASS_FP32, 1e-2, 30, None, heat32)
            h32 = host(heat32).astype(np.float64)
            assert np.abs(h32 / h32.max() - ref / ref.max()).max() <= 1e-3
        finally:
            gpu.grass_sparsifier_destroy(S)


def test_powerlaw_densify_round_matches_oracle(gpu, pl):
    import torch
    g, og, ot = pl
    r, t, sigma2, cap = 24, 3, 500.0, 2000
    h0s = [rng.gaussian_block(32, rng.STREAM_H0, g.n, r)]
    v0s = [rng.normal(32, rng.STREAM_V0, g.n)]
    res = oracle.densify(og, ot, h0s, v0s, sigma2, t, 1, 8, cap, record=True)
    with gpu_graph(g) as (ctx, tree, _):
        P = gpu.make_params(sigma2, r, t, 1, 8, cap, gpu.GRASS_FP64, 1e-12, 100)
        S, st = gpu.grass_densify(ctx, tree, P, dev(np.concatenate(h0s)), dev(np.concatenate(v0s)))
        try:
            mask = torch.empty(og.m, dtype=torch.uint8, device="cuda")
            gpu.grass_sparsifier_mask(ctx, S, mask)
            got = host(mask)
            d = st.as_dict()
            assert d["rounds"] == res.rounds
            assert d["lmin_est"][0] == pytest.approx(res.lmin[0], rel=1e-13)
            assert d["lmax_est"][0] == pytest.approx(res.lmax[0], rel=1e-8)
            for e in np.flatnonzero(got != res.in_s):
                assert _near_decision(res.trace, int(e)), int(e)
        finally:
            gpu.grass_sparsifier_destroy(S)


def _kappa(og, in_s):
    """Extreme generalized eigenvalues of (L_G, L_S) grounded at vertex 0,
    by ARPACK: lambda_max by Lanczos with L_S's factorisation, lambda_min by
    shift-invert about 0."""
    n = og.n

    def lap(mask):
        s = np.ones(og.m, bool) if mask is None else mask.astype(bool)
        L = sp.coo_matrix((np.concatenate([-og.ew[s]] * 2),
                           (np.concatenate([og.eu[s], og.ev[s]]), np.concatenate([og.ev[s], og.eu[s]]))),
                          shape=(n, n)).tocsr()
        L = L - sp.diags(np.asarray(L.sum(axis=1)).ravel())
        return L.tocsc()[1:, 1:]
    LG, LS = lap(None), lap(in_s)
    lmax = spla.eigsh(LG, k=1, M=LS, which="LA", return_eigenvectors=False, tol=1e-8)[0]
    lmin = spla.eigsh(LG, k=1, M=LS, sigma=0.0, which="LM", return_eigenvectors=False, tol=1e-8)[0]
    return lmax / lmin


@pytest.mark.parametrize("g_fn,sigma2,cap,r,t,rounds", [
    (lambda: graphs.grid3d_loguniform(20, 20, 20, seed=2), 200.0, 160, 16, 2, 3),
    (lambda: graphs.chung_lu(3000, seed=33), 500.0, 40, 24, 3, 2),
])
def test_fp32_condition_number_rule_larger(gpu, g_fn, sigma2, cap, r, t, rounds):
    import torch
    g = g_fn()
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    h0s = [rng.gaussian_block(5, rng.STREAM_H0 + k, g.n, r) for k in range(rounds)]
    v0s = [rng.normal(5, rng.STREAM_V0 + k, g.n) for k in range(rounds)]
    res = oracle.densify(og, ot, h0s, v0s, sigma2, t, rounds, 8, cap, 1e-12, 2000)
    k_ora = _kappa(og, res.in_s)
    with gpu_graph(g) as (ctx, tree, _):
        P = gpu.make_params(sigma2, r, t, rounds, 8, cap, gpu.GRASS_FP32, 1e-6, 300)
        S, st = gpu.grass_densify(ctx, tree, P, dev(np.concatenate(h0s)), dev(np.concatenate(v0s)))
        try:
            in_s = torch.empty(og.m, dtype=torch.uint8, device="cuda")
            gpu.grass_sparsifier_mask(ctx, S, in_s)
            k_gpu = _kappa(og, host(in_s))
        finally:
            gpu.grass_sparsifier_destroy(S)
    if k_ora <= sigma2:
        assert k_gpu <= sigma2, (k_gpu, k_ora)
    else:
        assert k_gpu <= 1.05 * k_ora, (k_gpu, k_ora)
