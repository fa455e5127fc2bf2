"""The serving form: requests admitted by device-memory footprint and run
concurrently on one GPU, each with its own device-resident state.

* every request's result is the same alone (one slot, one at a time) and in
  the mix (four slots, all submitted at once) -- bit for bit, since launch
  shapes depend on the request alone -- and equals the direct API path;
* every solution meets its tolerance, checked in FP64 on the host;
* admission honours the budget: with room for two requests at most, no
  more than two run at once; a request larger than the budget is refused.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from synth import graphs, rng
from tests.gpu_util import dev, gpu_graph, host

pytestmark = pytest.mark.gpu

R, T, ROUNDS = 8, 2, 2


def _requests():
    gs = [graphs.power_grid(60, 5), graphs.grid2d_uniform(90, 70, seed=3),
          graphs.power_grid(150, 6), graphs.grid3d_loguniform(20, 20, 20, seed=2),
          graphs.power_grid(40, 7), graphs.grid2d_uniform(200, 120, seed=4)]
    out = []
    for i, g in enumerate(gs):
        h0 = np.concatenate([rng.gaussian_block(30 + i, rng.STREAM_H0 + k, g.n, R) for k in range(ROUNDS)])
        v0 = np.concatenate([rng.normal(30 + i, rng.STREAM_V0 + k, g.n) for k in range(ROUNDS)])
        b = rng.normal(30 + i, rng.STREAM_RHS, g.n)
        out.append((g, h0, v0, b))
    return out


def _params(gpu):
    return gpu.make_params(100.0, R, T, ROUNDS, 8, 0, gpu.GRASS_FP32, 1e-2, 30)


PCG = dict(tol=1e-3, maxit=5000, pcg_prec=1, refine_tol=1e-3, pcg_inner_tol=1e-2, pcg_inner_maxit=1)


def _serve(gpu, reqs, slots, budget=0, one_at_a_time=False):
    srv = gpu.Server(0, slots, budget)
    try:
        xs, res = [], []
        tickets = []
        for g, h0, v0, b in reqs:
            x = np.full(g.n, np.nan)
            t = srv.submit(g.rowptr, g.col, g.val, h0, v0, b, x, _params(gpu), **PCG)
            if one_at_a_time:
                res.append(srv.wait(t))
            else:
                tickets.append(t)
            xs.append(x)
        for t in tickets:
            res.append(srv.wait(t))
        return xs, res, srv.stats()
    finally:
        srv.close()


def _rel_resid(g, x, b):
    A = sp.csr_matrix((g.val, g.col, g.rowptr), shape=(g.n, g.n))
    return np.linalg.norm(b - A @ x) / np.linalg.norm(b)


def test_same_alone_and_in_the_mix(gpu):
    reqs = _requests()
    x1, r1, s1 = _serve(gpu, reqs, slots=1, one_at_a_time=True)
    x4, r4, s4 = _serve(gpu, reqs, slots=4)
    assert s1["max_running"] == 1
    assert s4["max_running"] >= 2          # they did overlap
    for i, (g, h0, v0, b) in enumerate(reqs):
        assert r1[i].status == 0 and r4[i].status == 0, (r1[i].error, r4[i].error)
        assert _rel_resid(g, x1[i], b) <= 1e-3
        assert np.array_equal(x1[i], x4[i]), i
        assert r1[i].solve.iters == r4[i].solve.iters
        assert r1[i].sparsify.added == r4[i].sparsify.added
        assert r1[i].sparsify.rounds == r4[i].sparsify.rounds


def test_served_result_equals_direct_api(gpu):
    import torch
    g, h0, v0, b = _requests()[2]
    xs, res, _ = _serve(gpu, [(g, h0, v0, b)], slots=2)
    with gpu_graph(g) as (ctx, tree, _):
        S, st = gpu.grass_densify(ctx, tree, _params(gpu), dev(h0), dev(v0))
        try:
            x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
            s, ps = gpu.grass_pcg_solve(ctx, S, dev(b), x, PCG["tol"], PCG["maxit"], PCG["pcg_prec"],
                                        PCG["refine_tol"], PCG["pcg_inner_tol"], PCG["pcg_inner_maxit"])
        finally:
            gpu.grass_sparsifier_destroy(S)
    assert s == 0 and st.added == res[0].sparsify.added
    assert np.array_equal(host(x), xs[0])


def test_admission_by_footprint(gpu):
    reqs = _requests()
    fps = [gpu.grass_server_footprint(g.n, g.col.shape[0], R, ROUNDS) for g, *_ in reqs]
    budget = 2 * max(fps) + 1          # two of the largest fit, three never do
    xs, res, st = _serve(gpu, reqs, slots=4, budget=budget)
    assert st["max_running"] <= 2
    for (g, h0, v0, b), x, r in zip(reqs, xs, res):
        assert r.status == 0 and r.footprint_bytes > 0 and r.t_admit >= r.t_submit
        assert r.t_done >= r.t_admit and r.in_flight_at_admit <= 2
        assert _rel_resid(g, x, b) <= 1e-3
    # larger than the whole budget: refused at submission
    srv = gpu.Server(0, 1, min(fps) // 2)
    try:
        g, h0, v0, b = reqs[0]
        with pytest.raises(gpu.GrassError) as e:
            srv.submit(g.rowptr, g.col, g.val, h0, v0, b, np.zeros(g.n), _params(gpu), **PCG)
        assert e.value.status == gpu.GRASS_ERR_OOM
    finally:
        srv.close()


def test_footprint_bounds_measured_use(gpu):
    import torch
    g, h0, v0, b = _requests()[5]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    peak = [0]
    srv = gpu.Server(0, 1, 0)
    try:
        x = np.zeros(g.n)
        t = srv.submit(g.rowptr, g.col, g.val, h0, v0, b, x, _params(gpu), **PCG)
        import time
        while True:
            peak[0] = max(peak[0], free0 - torch.cuda.mem_get_info()[0])
            if srv.stats()["running"] == 0 and srv.stats()["queued"] == 0:
                break
            time.sleep(0.0005)
        r = srv.wait(t)
    finally:
        srv.close()
    assert r.status == 0
    # sampled peak (context + request) stays below the reserved footprint
    assert peak[0] <= r.footprint_bytes, (peak[0], r.footprint_bytes)
