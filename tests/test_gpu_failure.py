"""Failure detection on the GPU without faulting it: every grid-barrier wait
is bounded; a wait that runs out ends the kernel and the call returns
GRASS_ERR_TIMEOUT, after which the context still works."""
import numpy as np
import pytest

import oracle
from synth import graphs, rng
from tests.gpu_util import dev, gpu_graph, host

pytestmark = pytest.mark.gpu


def test_barrier_wait_runs_out_and_context_recovers(gpu):
    import torch
    # large enough that the solve's first rounds run across the grid (a few
    # thousand vertices fit in the single-block tail, which has no barrier)
    g = graphs.grid2d_uniform(120, 100, seed=61)
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    B = rng.gaussian_block(61, 1, g.n, 8)
    B -= B.mean(axis=0)
    ref = oracle.tree_solve(og, ot, B)
    with gpu_graph(g) as (ctx, tree, _):
        Bd = dev(B)
        X = torch.empty_like(Bd)
        # every barrier waits for a block that never comes: the wait must run out
        gpu.grass_ctx_set_wait_limit(ctx, 2000, 1)
        with pytest.raises(gpu.GrassError) as ei:
            gpu.grass_tree_solve(ctx, tree, 0, 8, gpu.GRASS_FP64, Bd, X)
        assert ei.value.status == gpu.GRASS_ERR_TIMEOUT
        assert "wait" in gpu.grass_last_error(ctx)
        # the same through the densification loop
        P = gpu.make_params(100.0, 8, 2, 1, 4, 0, gpu.GRASS_FP64, 1e-10, 100)
        with pytest.raises(gpu.GrassError) as ei:
            gpu.grass_densify(ctx, tree, P, dev(rng.gaussian_block(1, 2, g.n, 8)),
                              dev(rng.normal(1, 3, g.n)))
        assert ei.value.status == gpu.GRASS_ERR_TIMEOUT
        # back to normal limits: the context is usable and the result is right
        gpu.grass_ctx_set_wait_limit(ctx, 0, 0)
        gpu.grass_tree_solve(ctx, tree, 0, 8, gpu.GRASS_FP64, Bd, X)
        assert np.abs(host(X) - ref).max() <= 1e-10 * np.abs(ref).max()


def test_pcg_iteration_cap_reports_not_converged(gpu):
    import torch
    g = graphs.config_small_grid()
    b = rng.normal(1, rng.STREAM_RHS, g.n)
    with gpu_graph(g) as (ctx, tree, _):
        S = gpu.grass_sparsifier_create(ctx, tree)
        try:
            x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
            status, st = gpu.grass_pcg_solve(ctx, S, dev(b), x, 1e-10, 1, gpu.GRASS_FP64)
            assert status == gpu.GRASS_ERR_NOT_CONVERGED
            assert st.iters == 1 and st.rel_resid_fp64 > 1e-10
            assert np.isfinite(host(x)).all()
        finally:
            gpu.grass_sparsifier_destroy(S)
