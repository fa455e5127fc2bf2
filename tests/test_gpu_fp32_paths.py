"""FP32 paths of the fused Krylov kernels against the oracle, on sizes that
leave remainders:

* the 16-byte element loops: one column walks n in chunks of four (n mod 4
  elements left over: n = 1073, 1287, 3001); r = 4, 8, 16, 32 columns walk
  the n x r array in chunks, four fixed columns per thread;
* the two-row Laplacian products, which load four entries of a row at a
  time (3D grid rows have six; the power-law graph's hubs have hundreds);
* the inner CG in both forms (scan form and elimination rounds) and the
  fused PCG with and without off-tree edges in the sparsifier, and its
  closed-form single inner step on FP64 vectors.

Tolerances: FP32 vectors with float-pair dot products reach a relative
residual of 1e-6 in the inner solves, so an embedding's heats, normalised
by their maximum, agree with the oracle's (FP64, inner tolerance 1e-13) to
well inside 2e-3; lambda_max (a Rayleigh quotient after eight power steps)
to 1e-4; a PCG solve is judged by its own FP64 residual.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from synth import graphs, rng
from tests.gpu_util import dev, gpu_graph, host

pytestmark = pytest.mark.gpu

HEAT32_TOL = 2e-3     # per edge, relative to heat_max


def _with_extra(og, ot, every):
    in_s = ot.in_tree.copy()
    off = np.flatnonzero(in_s == 0)
    in_s[off[::every]] = 1
    return in_s, np.flatnonzero((in_s == 1) & (ot.in_tree == 0)).astype(np.int64)


# the scan form applies to one column only: r = 1 runs with it and without
@pytest.mark.parametrize("r,euler", [(1, 1), (1, 0), (2, 1), (4, 1), (8, 1), (16, 1), (24, 1), (32, 1)])
def test_fp32_embedding_through_inner_cg(gpu, r, euler):
    import torch
    g = graphs.grid2d_uniform(37, 29, seed=11)          # n = 1073
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    in_s, add = _with_extra(og, ot, 5)
    h0 = rng.gaussian_block(71 + r, rng.STREAM_H0, g.n, r)
    H_ref = oracle.embed(og, ot, in_s, h0, 2, 1e-13, 3000)
    hv_ref, off_ref = oracle.heat(og, in_s, H_ref)
    with gpu_graph(g) as (ctx, tree, _):
        gpu.grass_ctx_set_param(ctx, "euler_solve", euler)
        S = gpu.grass_sparsifier_create(ctx, tree)
        try:
            gpu.grass_sparsifier_add(ctx, S, dev(add))
            heat = torch.empty(off_ref.shape[0], dtype=torch.float32, device="cuda")
            gpu.grass_embed(ctx, S, dev(h0), r, 2, gpu.GRASS_FP32, 1e-6, 3000, None, heat)
            hv = host(heat).astype(np.float64)
        finally:
            gpu.grass_sparsifier_destroy(S)
    err = np.abs(hv / hv.max() - hv_ref / hv_ref.max()).max()
    assert err <= HEAT32_TOL, err


def _sdd(g, d=1e-3):
    """g with d added to every diagonal entry (D = d I)."""
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    val = g.val.copy()
    val[g.col == rows] += d
    return graphs.Graph(g.name + "_sdd", g.n, g.rowptr, g.col, val)


def _pcg_cases():
    return [graphs.grid3d_loguniform(13, 11, 9, seed=12),    # n = 1287, rows of 6
            graphs.ring_chords(3001, seed=13),               # n = 3001
            _sdd(graphs.chung_lu(6001, seed=6))]             # hubs: rows of up to 245


@pytest.mark.parametrize("gi", range(3))
@pytest.mark.parametrize("extra", [False, True])
def test_fp32_pcg_ragged_sizes(gpu, gi, extra):
    import torch
    g = _pcg_cases()[gi]
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    b = rng.normal(81 + gi, rng.STREAM_RHS, g.n)
    tol = 1e-6
    with gpu_graph(g) as (ctx, tree, _):
        S = gpu.grass_sparsifier_create(ctx, tree)
        try:
            if extra:
                _, add = _with_extra(og, ot, 3)
                gpu.grass_sparsifier_add(ctx, S, dev(add))
            x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
            status, st = gpu.grass_pcg_solve(ctx, S, dev(b), x, tol, 20000, gpu.GRASS_FP32,
                                             1e-3, 1e-2, 1)
            assert status == gpu.GRASS_OK
        finally:
            gpu.grass_sparsifier_destroy(S)
    A = sp.csr_matrix((g.val, g.col, g.rowptr), shape=(g.n, g.n))
    xr = host(x)
    rel = np.linalg.norm(b - A @ xr) / np.linalg.norm(b)
    assert rel <= tol and st.rel_resid_fp64 == pytest.approx(rel, rel=1e-6)


@pytest.mark.parametrize("gi", range(3))
def test_fp64_pcg_one_inner_step(gpu, gi):
    """FP64 vectors with one inner step per outer iteration: the closed-form
    step on doubles (one element per step, no 16-byte chunks)."""
    import torch
    g = _pcg_cases()[gi]
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    b = rng.normal(85 + gi, rng.STREAM_RHS, g.n)
    tol = 1e-9
    with gpu_graph(g) as (ctx, tree, _):
        S = gpu.grass_sparsifier_create(ctx, tree)
        try:
            _, add = _with_extra(og, ot, 3)
            gpu.grass_sparsifier_add(ctx, S, dev(add))
            x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
            status, st = gpu.grass_pcg_solve(ctx, S, dev(b), x, tol, 20000, gpu.GRASS_FP64,
                                             1e-3, 1e-2, 1)
            assert status == gpu.GRASS_OK and st.inner_iters == st.iters
        finally:
            gpu.grass_sparsifier_destroy(S)
    A = sp.csr_matrix((g.val, g.col, g.rowptr), shape=(g.n, g.n))
    rel = np.linalg.norm(b - A @ host(x)) / np.linalg.norm(b)
    assert rel <= tol


@pytest.mark.parametrize("euler", [1, 0])
def test_fp32_lambda_max_matches_oracle(gpu, euler):
    g = graphs.grid3d_loguniform(13, 11, 9, seed=12)        # n = 1287
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    in_s, add = _with_extra(og, ot, 7)
    v0 = rng.normal(91, rng.STREAM_V0, g.n)
    ref = oracle.lambda_max_est(og, ot, in_s, v0, 8, 1e-13, 3000)
    with gpu_graph(g) as (ctx, tree, _):
        gpu.grass_ctx_set_param(ctx, "euler_solve", euler)
        S = gpu.grass_sparsifier_create(ctx, tree)
        try:
            gpu.grass_sparsifier_add(ctx, S, dev(add))
            lmax = gpu.grass_lambda_max(ctx, S, dev(v0), 8, gpu.GRASS_FP32, 1e-6, 3000)
        finally:
            gpu.grass_sparsifier_destroy(S)
    assert lmax == pytest.approx(ref, rel=1e-4)
