"""The sparsifier's aggregation multigrid (the sparsifier solver of Sec.
IV-C-1 / IV-D step 1): as the PCG preconditioner of A = L_G + D (Sec. V-A)
and for the lambda_max estimate's solves with L_S.

* PCG with the V-cycle of L_S + D reaches the tolerance, judged by an
  independent FP64 residual, in FP64 and in FP32 with FP64 refinement, in
  fewer iterations than the tree preconditioner (including a unit-weight
  mesh, where every matching choice is a tie);
* the lambda_max estimate with multigrid-CG solves equals the oracle's
  (tight inner solves on both sides) to 1e-9;
* a pure Laplacian (D = 0, singular): the partitioner's solves converge;
* the multigrid PCG as one cooperative kernel per pass equals the form with
  one launch per level step.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from synth import graphs, rng
from tests.gpu_util import dev, gpu_graph, host

pytestmark = pytest.mark.gpu


def _with_extra(gpu, ctx, tree, og, ot, every):
    S = gpu.grass_sparsifier_create(ctx, tree)
    in_s = ot.in_tree.copy()
    in_s[np.flatnonzero(in_s == 0)[::every]] = 1
    add = np.flatnonzero((in_s == 1) & (ot.in_tree == 0)).astype(np.int64)
    gpu.grass_sparsifier_add(ctx, S, dev(add))
    return S, in_s


@pytest.mark.parametrize("which", ["grid3d", "powergrid", "powerlaw", "unitmesh"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_amg_preconditioned_pcg(gpu, which, prec):
    import torch
    g = {"grid3d": lambda: graphs.grid3d_loguniform(30, 27, 25, seed=101),
         "powergrid": lambda: graphs.power_grid(150, seed=102),
         "powerlaw": lambda: graphs.chung_lu(30000, seed=103),
         # all weights equal: the matching's ties decide every choice
         "unitmesh": lambda: graphs.grid((170, 160), None, 1e-3)}[which]()
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    if not np.any(og.D > 0):
        pytest.skip("pure Laplacian: covered by the partition test")
    b = rng.normal(101, rng.STREAM_RHS, g.n)
    A = sp.csr_matrix((g.val, g.col, g.rowptr), shape=(g.n, g.n))
    tol = 1e-8
    P = gpu.GRASS_FP64 if prec == "fp64" else gpu.GRASS_FP32
    with gpu_graph(g) as (ctx, tree, _):
        S, _ = _with_extra(gpu, ctx, tree, og, ot, 10)
        try:
            x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
            st0, s0 = gpu.grass_pcg_solve(ctx, S, dev(b), x, tol, 20000, P, 1e-2, 1e-2, 0)
            gpu.grass_ctx_set_param(ctx, "pcg_precond", 1)
            x.zero_()
            st1, s1 = gpu.grass_pcg_solve(ctx, S, dev(b), x, tol, 20000, P, 1e-2, 1e-2, 0)
            assert st1 == gpu.GRASS_OK
            rel = np.linalg.norm(b - A @ host(x)) / np.linalg.norm(b)
            assert rel <= tol and s1.rel_resid_fp64 == pytest.approx(rel, rel=1e-6)
            assert s1.iters < s0.iters, (s1.iters, s0.iters)
        finally:
            gpu.grass_sparsifier_destroy(S)


@pytest.mark.parametrize("which", ["grid3d", "powergrid", "unitmesh", "one_level"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fused_multigrid_pcg_matches_launch_form(gpu, which, prec):
    """The multigrid PCG as one cooperative kernel per pass against the same
    iteration run as one launch per level step (CUDA graph replay): the same
    V-cycle, so the iteration counts agree within 2 and the solutions within
    the tolerance, for every split of the levels between the grid and
    block 0 (none but the coarsest solve, 4096, all of them) and between
    thread-per-row and warp-per-row phases;
    "one_level" has at most 256 vertices, so the V-cycle is the coarsest
    dense solve alone."""
    import torch
    g = {"grid3d": lambda: graphs.grid3d_loguniform(30, 27, 25, seed=101),
         "powergrid": lambda: graphs.power_grid(150, seed=102),
         "unitmesh": lambda: graphs.grid((170, 160), None, 1e-3),
         "one_level": lambda: graphs.grid2d_uniform(15, 16, seed=106, D=1e-3)}[which]()
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    b = rng.normal(107, rng.STREAM_RHS, g.n)
    A = sp.csr_matrix((g.val, g.col, g.rowptr), shape=(g.n, g.n))
    tol = 1e-8
    P = gpu.GRASS_FP64 if prec == "fp64" else gpu.GRASS_FP32
    with gpu_graph(g) as (ctx, tree, _):
        S, _ = _with_extra(gpu, ctx, tree, og, ot, 10)
        try:
            gpu.grass_ctx_set_param(ctx, "pcg_precond", 1)
            gpu.grass_ctx_set_param(ctx, "amg_fused", 0)
            x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
            st0, s0 = gpu.grass_pcg_solve(ctx, S, dev(b), x, tol, 20000, P, 1e-2, 1e-2, 0)
            assert st0 == gpu.GRASS_OK
            x0 = host(x)
            gpu.grass_ctx_set_param(ctx, "amg_fused", 1)
            for tail, warp in ((0, 0), (0, 4096), (0, 1 << 40), (4096, 4096), (1 << 40, 0)):
                gpu.grass_ctx_set_param(ctx, "amg_tail_n", tail)
                gpu.grass_ctx_set_param(ctx, "amg_warp_n", warp)
                x.zero_()
                st1, s1 = gpu.grass_pcg_solve(ctx, S, dev(b), x, tol, 20000, P, 1e-2, 1e-2, 0)
                assert st1 == gpu.GRASS_OK
                x1 = host(x)
                rel = np.linalg.norm(b - A @ x1) / np.linalg.norm(b)
                assert rel <= tol and s1.rel_resid_fp64 == pytest.approx(rel, rel=1e-6)
                assert abs(s1.iters - s0.iters) <= 2, (tail, warp, s1.iters, s0.iters)
                assert np.linalg.norm(x1 - x0) <= 1e-6 * np.linalg.norm(x0), (tail, warp)
        finally:
            gpu.grass_sparsifier_destroy(S)


@pytest.mark.parametrize("which", ["grid3d", "powergrid"])
def test_warp_setup_builds_the_same_hierarchy(gpu, which):
    """The setup's warp forms (matching candidates, coarse-row counts and
    fill, one warp per vertex on small levels) build the hierarchy the
    thread forms build: the multigrid PCG on it then runs the same
    iterations to the same FP64 solution, bit for bit."""
    import torch
    g = {"grid3d": lambda: graphs.grid3d_loguniform(30, 27, 25, seed=101),
         "powergrid": lambda: graphs.power_grid(150, seed=102)}[which]()
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    b = rng.normal(108, rng.STREAM_RHS, g.n)
    xs, its = [], []
    for warp_setup in (0, 1 << 40):
        with gpu_graph(g) as (ctx, tree, _):
            gpu.grass_ctx_set_param(ctx, "amg_warp_setup_n", warp_setup)
            gpu.grass_ctx_set_param(ctx, "pcg_precond", 1)
            S, _ = _with_extra(gpu, ctx, tree, og, ot, 10)
            try:
                x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
                st, s = gpu.grass_pcg_solve(ctx, S, dev(b), x, 1e-8, 20000, gpu.GRASS_FP64, 1e-2,
                                            1e-2, 0)
                assert st == gpu.GRASS_OK
                xs.append(host(x))
                its.append(s.iters)
            finally:
                gpu.grass_sparsifier_destroy(S)
    assert its[0] == its[1]
    assert np.array_equal(xs[0], xs[1])


def test_amg_lambda_max_matches_oracle(gpu):
    g = graphs.grid2d_uniform(60, 45, seed=104)
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    v0 = rng.normal(104, rng.STREAM_V0, g.n)
    with gpu_graph(g) as (ctx, tree, _):
        S, in_s = _with_extra(gpu, ctx, tree, og, ot, 6)
        try:
            gpu.grass_ctx_set_param(ctx, "lmax_amg", 1)
            lm = gpu.grass_lambda_max(ctx, S, dev(v0), 8, gpu.GRASS_FP64, 1e-12, 500)
            ref = oracle.lambda_max_est(og, ot, in_s, v0, 8, 1e-13, 3000)
            assert lm == pytest.approx(ref, rel=1e-9)
        finally:
            gpu.grass_sparsifier_destroy(S)


def test_amg_densify_certifies_and_matches_oracle(gpu):
    import torch
    g = graphs.grid3d_loguniform(12, 12, 12, seed=2)
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    rounds, r, sigma2, cap = 3, 16, 20.0, 60
    h0s = [rng.gaussian_block(9, rng.STREAM_H0 + k, g.n, r) for k in range(rounds)]
    v0s = [rng.normal(9, rng.STREAM_V0 + k, g.n) for k in range(rounds)]
    res = oracle.densify(og, ot, h0s, v0s, sigma2, 2, rounds, 8, cap, 1e-13, 3000)
    with gpu_graph(g) as (ctx, tree, _):
        gpu.grass_ctx_set_param(ctx, "lmax_amg", 1)
        P = gpu.make_params(sigma2, r, 2, rounds, 8, cap, gpu.GRASS_FP64, 1e-13, 3000)
        S, st = gpu.grass_densify(ctx, tree, P, dev(np.concatenate(h0s)), dev(np.concatenate(v0s)))
        try:
            d = st.as_dict()
            assert d["rounds"] == res.rounds
            assert all(c == 0 for c in d["lmax_capped"])
            for k in range(len(res.lmax)):
                assert d["lmax_est"][k] == pytest.approx(res.lmax[k], rel=1e-8)
        finally:
            gpu.grass_sparsifier_destroy(S)


def test_amg_partition_on_a_pure_laplacian(gpu):
    import torch
    g = graphs.grid2d_uniform(200, 150, seed=105, D=0.0)
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    x0 = dev(rng.normal(105, 1, g.n))
    with gpu_graph(g) as (ctx, tree, _):
        S, _ = _with_extra(gpu, ctx, tree, og, ot, 8)
        try:
            s_tree = torch.empty(g.n, dtype=torch.uint8, device="cuda")
            st0, f0 = gpu.grass_fiedler(ctx, S, x0, 4, 1e-8, 100000, gpu.GRASS_FP64, 0, None, s_tree)
            gpu.grass_ctx_set_param(ctx, "pcg_precond", 1)
            s_amg = torch.empty_like(s_tree)
            st1, f1 = gpu.grass_fiedler(ctx, S, x0, 4, 1e-8, 100000, gpu.GRASS_FP64, 0, None, s_amg)
            assert st0 == gpu.GRASS_OK and st1 == gpu.GRASS_OK and f1.worst_rel_resid <= 1e-8
            assert f1.pcg_iters < f0.pcg_iters, (f1.pcg_iters, f0.pcg_iters)
            assert np.mean(host(s_tree) == host(s_amg)) >= 0.999
        finally:
            gpu.grass_sparsifier_destroy(S)
