"""grass_tree_solve_noalloc, the tree solve without device allocation, against
grass_tree_solve on the same inputs, through the C ABI.

The no-allocation entry keeps its scratch in one array per device that every
call shares and that holds the previous call's contents, so each case makes
two calls in a row (different right-hand sides) and checks both.  The file
is named to be collected last: it must pass alone in a fresh process (the
first call does the per-device set-up) and after every other test.
"""
import numpy as np
import pytest

from synth import graphs, rng
from tests.gpu_util import dev, gpu_graph, host

pytestmark = pytest.mark.gpu

SOLVE_TOL = 1e-10      # relative to max |x|, as for the FP64 tree-solve parity tests
SOLVE_TOL_FP32 = 1e-5  # FP32: same kernel arithmetic, so far tighter than FP32 vs FP64


def _graphs():
    # 12000 vertices: more than the shared-memory tail, so the grid barriers
    # (whose counter lives in the shared array) run; 64000 on the 3D grid
    return [graphs.grid2d_uniform(120, 100, seed=5), graphs.grid3d_loguniform(40, 40, 40, seed=6)]


@pytest.mark.parametrize("gi", [0, 1])
@pytest.mark.parametrize("prec,r", [("fp64", 8), ("fp64", 1), ("fp32", 16), ("fp32", 32)])
def test_noalloc_matches_tree_solve_two_calls(gpu, gi, prec, r):
    import torch
    g = _graphs()[gi]
    P = gpu.GRASS_FP64 if prec == "fp64" else gpu.GRASS_FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = SOLVE_TOL if prec == "fp64" else SOLVE_TOL_FP32
    with gpu_graph(g) as (ctx, tree, _):
        for with_D in (0, 1):
            for call in range(2):
                B = rng.gaussian_block(40 + 2 * gi + with_D, 10 + call, g.n, r)
                Bd = dev(B, dt)
                X_ref = torch.empty_like(Bd)
                gpu.grass_tree_solve(ctx, tree, with_D, r, P, Bd, X_ref)   # builds L_T + D once
                X = torch.full_like(Bd, float("nan"))
                gpu.grass_tree_solve_noalloc(ctx, tree, with_D, r, P, Bd, X)
                ref = host(X_ref).astype(np.float64)
                x = host(X).astype(np.float64)
                assert np.all(np.isfinite(x)), (with_D, call)
                assert np.abs(x - ref).max() <= tol * np.abs(ref).max(), (with_D, call)
                # in place (B and X alias), as grass_tree_solve allows
                Y = Bd.clone()
                gpu.grass_tree_solve_noalloc(ctx, tree, with_D, r, P, Y, Y)
                assert np.abs(host(Y).astype(np.float64) - ref).max() <= tol * np.abs(ref).max()


def test_noalloc_rejects_what_it_cannot_serve(gpu):
    import torch
    g = graphs.grid2d_uniform(30, 20, seed=5)
    with gpu_graph(g) as (ctx, tree, _):
        B = dev(rng.gaussian_block(50, 1, g.n, 4))
        X = torch.empty_like(B)
        # L_T + D not built yet: building it would allocate
        with pytest.raises(gpu.GrassError) as e:
            gpu.grass_tree_solve_noalloc(ctx, tree, 1, 4, gpu.GRASS_FP64, B, X)
        assert e.value.status == gpu.GRASS_ERR_INVALID
        assert "with_D=1" in str(e.value)
        with pytest.raises(gpu.GrassError) as e:
            gpu.grass_tree_solve_noalloc(ctx, tree, 0, 3, gpu.GRASS_FP64, B, X)
        assert e.value.status == gpu.GRASS_ERR_INVALID
        # still usable after the rejections, and equal to the allocating solve
        X_ref = torch.empty_like(B)
        gpu.grass_tree_solve(ctx, tree, 0, 4, gpu.GRASS_FP64, B, X_ref)
        gpu.grass_tree_solve_noalloc(ctx, tree, 0, 4, gpu.GRASS_FP64, B, X)
        ref = host(X_ref)
        assert np.abs(host(X) - ref).max() <= SOLVE_TOL * np.abs(ref).max()


def test_noalloc_leaves_device_memory_unchanged(gpu):
    """Once the kernels are loaded (the first call) and the L_T + D factor
    exists, further calls take no device memory: the free memory the driver
    reports is the same before and after them."""
    import torch
    g = graphs.grid3d_loguniform(40, 40, 40, seed=6)
    with gpu_graph(g) as (ctx, tree, _):
        B = dev(rng.gaussian_block(60, 1, g.n, 8))
        X = torch.empty_like(B)
        gpu.grass_tree_solve(ctx, tree, 1, 8, gpu.GRASS_FP64, B, X)      # builds L_T + D
        for with_D in (0, 1):
            gpu.grass_tree_solve_noalloc(ctx, tree, with_D, 8, gpu.GRASS_FP64, B, X)   # warm
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for with_D in (0, 1, 0, 1):
            gpu.grass_tree_solve_noalloc(ctx, tree, with_D, 8, gpu.GRASS_FP64, B, X)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0


def test_noalloc_bounded_wait_runs_out_and_recovers(gpu):
    """The barrier waits of the no-allocation solve are bounded like those of
    grass_tree_solve: with the context's test hold on, every wait runs out,
    the call returns GRASS_ERR_TIMEOUT, and the next normal call is right."""
    import torch
    g = graphs.grid2d_uniform(120, 100, seed=5)
    with gpu_graph(g) as (ctx, tree, _):
        B = dev(rng.gaussian_block(61, 1, g.n, 4))
        X_ref = torch.empty_like(B)
        gpu.grass_tree_solve(ctx, tree, 0, 4, gpu.GRASS_FP64, B, X_ref)
        X = torch.empty_like(B)
        gpu.grass_ctx_set_wait_limit(ctx, 2000, 1)
        with pytest.raises(gpu.GrassError) as e:
            gpu.grass_tree_solve_noalloc(ctx, tree, 0, 4, gpu.GRASS_FP64, B, X)
        assert e.value.status == gpu.GRASS_ERR_TIMEOUT
        gpu.grass_ctx_set_wait_limit(ctx, 0, 0)
        gpu.grass_tree_solve_noalloc(ctx, tree, 0, 4, gpu.GRASS_FP64, B, X)
        ref = host(X_ref)
        assert np.abs(host(X) - ref).max() <= SOLVE_TOL * np.abs(ref).max()
