#!/usr/bin/env python3
"""Benchmark of the GB300 sparsify-and-solve path (GRASS, arXiv 1911.04382).

One step = the whole hot path over one synthetic SDD matrix resident in HBM:
validate + extract edges, maximum spanning tree + elimination schedule,
densification rounds (lambda estimates, t-step power iteration over r random
vectors, Joule heat, threshold filter with per-round cap, sparsifier
update), then the PCG solve of A = L_G + D preconditioned by the sparsifier.

Metric: off-tree edges embedded per second = (sum over rounds of the edges
outside the sparsifier that were embedded) / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...     # the CPU oracle, on host cores

Prints one JSON line (rank 0).  N > 1 (torchrun): independent replicas, one
per GPU, timing max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "off-tree edges embedded/s"
UNIT = "edges/s"

WORKLOADS = {
    # 100^3 7-point grid, log-uniform weights in [1e-2, 1e2], D = 1e-3 I
    # PCG inner budget: outer iterations stay ~400 for 1..32 inner CG
    # iterations (measured), so one inner iteration is the fastest setting
    "grid3d_100": dict(kind="grid3d", side=100, seed=2, r=16, t=2, sigma2=200.0, rounds=3,
                       lmax_iters=8, cap_frac=0.02, embed="fp32", inner_tol=1e-2, inner_maxit=30,
                       pcg="fp32", pcg_tol=1e-8, refine_tol=1e-2, pcg_inner_tol=1e-2,
                       pcg_inner_maxit=1, pcg_maxit=4000),
    # 64x64 5-point grid, w ~ U[1,10), D = 1e-3 I, plain FP64 method
    "grid2d_64": dict(kind="grid2d", side=64, seed=1, r=8, t=2, sigma2=100.0, rounds=1,
                      lmax_iters=8, cap_frac=0.0, embed="fp64", inner_tol=1e-10, inner_maxit=1000,
                      pcg="fp64", pcg_tol=1e-3, refine_tol=1e-2, pcg_inner_tol=1e-6,
                      pcg_inner_maxit=50, pcg_maxit=4000),
    # quick check of the same shape as grid3d_100
    "grid3d_40": dict(kind="grid3d", side=40, seed=2, r=16, t=2, sigma2=200.0, rounds=3,
                      lmax_iters=8, cap_frac=0.02, embed="fp32", inner_tol=1e-2, inner_maxit=30,
                      pcg="fp32", pcg_tol=1e-8, refine_tol=1e-2, pcg_inner_tol=1e-2,
                      pcg_inner_maxit=1, pcg_maxit=4000),
}

FAMILIES = {"spmm_g": 1, "spmm_s": 2, "heat": 3, "tree": 4, "cg": 5, "pcg": 6, "spmm_blk": 7}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def peak_hbm() -> float:
    """Measured copy bandwidth (GB/s), else the 6800 GB/s fallback."""
    return float(measured_peaks().get("hbm_gbs", 6800.0))


def make_inputs(w: dict):
    from synth import graphs, rng
    if w["kind"] == "grid3d":
        s = w["side"]
        g = graphs.grid3d_loguniform(s, s, s, w["seed"])
    else:
        g = graphs.grid2d_uniform(w["side"], w["side"], w["seed"])
    R = w["rounds"]
    h0 = np.concatenate([rng.gaussian_block(w["seed"], rng.STREAM_H0 + k, g.n, w["r"])
                         for k in range(R)])
    v0 = np.concatenate([rng.normal(w["seed"], rng.STREAM_V0 + k, g.n) for k in range(R)])
    b = rng.normal(w["seed"], rng.STREAM_RHS, g.n)
    return g, h0, v0, b


def describe(w: dict, g) -> str:
    if w["kind"] == "grid3d":
        s = w["side"]
        return (f"3D 7-point grid {s}x{s}x{s} ({g.n} nodes, {g.m} edges), w = 10^U(-2,2), "
                f"D = 1e-3 I; r={w['r']}, t={w['t']}, sigma^2={w['sigma2']:g}, "
                f"{w['rounds']} densification rounds; {w['embed'].upper()} embedding; "
                f"PCG {w['pcg'].upper()}{' + FP64 refinement' if w['pcg'] == 'fp32' else ''} "
                f"to {w['pcg_tol']:g}")
    s = w["side"]
    return (f"2D 5-point grid {s}x{s} ({g.n} nodes, {g.m} edges), w ~ U[1,10), D = 1e-3 I; "
            f"r={w['r']}, t={w['t']}, sigma^2={w['sigma2']:g}, {w['rounds']} round; "
            f"{w['embed'].upper()}; PCG to {w['pcg_tol']:g}")


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), p[4], p[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, _, f in rows for i in range(4) if f[i] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- reference arm (oracle)

def oracle_sample(w: dict, g, h0, v0):
    """The CPU oracle on a bounded sample of the step: edge extraction,
    Kruskal tree, round-1 lambda estimates, FP64 embedding over the same r
    vectors, heat and filter on the full matrix.  Returns (edges, seconds)."""
    import oracle
    t0 = time.perf_counter()
    og = oracle.from_graph(g)
    ot = oracle.build_tree(og)
    lmin = oracle.lambda_min_est(og, ot.in_tree)
    lmax = oracle.lambda_max_est(og, ot, ot.in_tree, v0[:g.n], w["lmax_iters"])
    H = oracle.embed(og, ot, None, h0[:g.n], w["t"])
    hv, off = oracle.heat(og, ot.in_tree, H)
    cap = int(w["cap_frac"] * g.n)
    oracle.filter_edges(hv, off, oracle.theta_sigma(w["sigma2"], lmin, lmax, w["t"]), cap)
    return int(off.shape[0]), time.perf_counter() - t0


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    g, h0, v0, b = make_inputs(w)
    for _ in range(args.warmup):
        oracle_sample(w, g, h0, v0)
    times, edges = [], 0
    for _ in range(args.steps):
        e, s = oracle_sample(w, g, h0, v0)
        edges = e
        times.append(s)
    ms = 1e3 * sum(times) / len(times)
    value = edges / (ms / 1e3)
    sample = ("per step: oracle extraction + Kruskal tree + round-1 lambda estimates + FP64 "
              "embedding/heat/filter of every off-tree edge on the full matrix (single thread)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": describe(w, g), "name": args.workload},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- kernel captures

KERNEL_SOURCES = ["paper_1911_04382_gb300/csrc/krylov.cu", "paper_1911_04382_gb300/csrc/solve.cu",
                  "paper_1911_04382_gb300/csrc/tree_solve.cuh",
                  "paper_1911_04382_gb300/csrc/common.cuh",
                  "paper_1911_04382_gb300/csrc/amg_fused.cu"]


def kernel_sources_hash(read=None) -> str:
    """Hash of the kernel sources' code: comments and blank lines removed,
    so a comment edit keeps a capture's record valid.  read(path) -> text
    (default: the working tree)."""
    import hashlib
    import re
    read = read or (lambda s: open(os.path.join(ROOT, s)).read())
    h = hashlib.sha256()
    for s in KERNEL_SOURCES:
        t = re.sub(r"/\*.*?\*/", "", read(s), flags=re.S)
        t = re.sub(r"//[^\n]*", "", t)
        h.update("\n".join(ln.rstrip() for ln in t.splitlines() if ln.strip()).encode())
    return h.hexdigest()[:16]


def profile_kernel(G, ctx, which, g, rp, col, val, v0d, w) -> int:
    """One warm and one timed launch of the fused inner CG (exactly 30
    iterations, r = 1 -- "cg" -- or r = 16 -- "cg16", one embedding step --,
    FP32, sparsifier = tree + every 197th off-tree edge), of the fused PCG
    ("pcg": tree solve and one inner step; "amgpcg": the multigrid V-cycle),
    or of the tree solve (r = 16, FP32); prints its algorithmic bytes."""
    import torch
    tree = G.grass_build_tree(ctx, rp, col, val, 0)
    if which in ("cg", "pcg", "cg16", "amgpcg"):
        S = G.grass_sparsifier_create(ctx, tree)
        _, moff = G.grass_sparsifier_info(S)
        ids = torch.empty(moff, dtype=torch.int64, device="cuda")
        G.grass_sparsifier_offtree(ctx, S, ids)
        G.grass_sparsifier_add(ctx, S, ids[::197].contiguous())
        if which == "cg":
            run = lambda: G.grass_lambda_max(ctx, S, v0d[:g.n], 1, G.GRASS_FP32, 0.0, 30)
            fam, units = G.GRASS_KF_CG, "30 iterations, r=1"
        elif which == "cg16":
            from synth import rng as _rng
            h16 = torch.from_numpy(_rng.gaussian_block(w["seed"], _rng.STREAM_H0, g.n, 16)).cuda()
            run = lambda: G.grass_embed(ctx, S, h16, 16, 1, G.GRASS_FP32, 0.0, 30)
            fam, units = G.GRASS_KF_CG, "30 iterations, r=16 (one embedding step)"
        else:
            bq = v0d[:g.n].contiguous()
            xq = torch.zeros(g.n, dtype=torch.float64, device="cuda")
            # one FP32 pass of exactly 30 outer iterations (tolerance out of reach);
            # "amgpcg": the fused multigrid PCG (the warm run builds the hierarchy)
            mg = which == "amgpcg"
            G.grass_ctx_set_param(ctx, "pcg_precond", 1 if mg else 0)
            run = lambda: G.grass_pcg_solve(ctx, S, bq, xq, 1e-30, 30, G.GRASS_FP32, 1e-20, 1e-2,
                                            0 if mg else 1)
            fam, units = G.GRASS_KF_PCG, ("30 outer iterations, one V-cycle each" if mg
                                          else "30 outer iterations, inner 1")
    else:
        B = torch.randn(g.n, 16, dtype=torch.float32, device="cuda")
        X = torch.empty_like(B)
        run = lambda: G.grass_tree_solve(ctx, tree, 0, 16, G.GRASS_FP32, B, X)
        fam, units = G.GRASS_KF_TREE, "one solve, r=16"
    run()
    G.grass_kernel_timing_enable(ctx, fam)
    run()
    ms, nl, by = G.grass_kernel_timing_read(ctx)
    print(json.dumps({"profile_kernel": which, "launches": nl, "ms": ms, "algorithmic_bytes": by,
                      "units": units, "sources": kernel_sources_hash()}), flush=True)
    return 0


# ---------------------------------------------------------------- 40M-unknown solve

SOLVE40M = dict(k=6325, seed=5, r=8, t=2, sigma2=100.0, rounds=2, lmax_iters=8, cap_frac=0.05,
                inner_tol=1e-2, inner_maxit=30, tol=1e-3, refine_tol=1e-3, pcg_inner_tol=1e-2,
                pcg_inner_maxit=1, maxit=5000)


def solve_40m(G, w=SOLVE40M) -> dict:
    """The 6325 x 6325 power-grid mesh (40,005,625 unknowns, ~2.0e8 stored
    entries, 1 % vias, pad loads): maximum spanning tree, densification and
    PCG to ||b - Ax|| <= 1e-3 ||b||, timed from the device-resident CSR to x
    (the paper's T_I includes the preconditioner's construction); e2e adds
    the copies of the CSR and b from pinned host memory and of x back.  The
    start blocks h0, v0 come from torch's seeded device generator."""
    import torch
    from synth import graphs, rng
    t0 = time.perf_counter()
    g = graphs.power_grid(w["k"], w["seed"])
    b = rng.normal(w["seed"], rng.STREAM_RHS, g.n)
    gen_s = time.perf_counter() - t0
    gen = torch.Generator(device="cuda").manual_seed(w["seed"])
    h0 = torch.randn(w["rounds"] * g.n * w["r"], generator=gen, device="cuda", dtype=torch.float64)
    v0 = torch.randn(w["rounds"] * g.n, generator=gen, device="cuda", dtype=torch.float64)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hp = [pin(g.rowptr), pin(g.col), pin(g.val), pin(b)]
    dv = [torch.empty_like(t, device="cuda") for t in hp]
    for d, h in zip(dv, hp):
        d.copy_(h)
    xh = torch.empty(g.n, dtype=torch.float64).pin_memory()
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    P = G.make_params(w["sigma2"], w["r"], w["t"], w["rounds"], w["lmax_iters"],
                      int(w["cap_frac"] * g.n), G.GRASS_FP32, w["inner_tol"], w["inner_maxit"])
    ctx = G.grass_ctx_create()
    out = {}

    def once(copy_in: bool):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if copy_in:
            for d, h in zip(dv, hp):
                d.copy_(h, non_blocking=True)
        t1 = time.perf_counter()
        tree = G.grass_build_tree(ctx, dv[0], dv[1], dv[2], 0)
        t2 = time.perf_counter()
        S, st = G.grass_densify(ctx, tree, P, h0, v0)
        t3 = time.perf_counter()
        s, ps = G.grass_pcg_solve(ctx, S, dv[3], x, w["tol"], w["maxit"], G.GRASS_FP32,
                                  w["refine_tol"], w["pcg_inner_tol"], w["pcg_inner_maxit"])
        t4 = time.perf_counter()
        if copy_in:
            xh.copy_(x)
        torch.cuda.synchronize()
        t5 = time.perf_counter()
        n_s, _ = G.grass_sparsifier_info(S)
        G.grass_sparsifier_destroy(S)
        G.grass_tree_destroy(tree)
        return dict(total=t5 - t0, tree=t2 - t1, densify=t3 - t2, pcg=t4 - t3, status=s,
                    iters=ps.iters, rel=ps.rel_resid_fp64, rounds=st.rounds, added=st.added,
                    lmax=list(st.lmax_est[:st.rounds + 1]), n_s=n_s,
                    capped=list(st.lmax_capped[:st.rounds + 1]),
                    stopped=bool(st.stopped_similar))

    try:
        once(False)                                  # warm (allocations, first launches)
        a = once(False)
        e = once(True)
        # the same solve with the lambda_max estimate's solves by
        # multigrid-preconditioned CG (lmax_amg): a converged estimate may
        # let the stop test end densification early
        G.grass_ctx_set_param(ctx, "lmax_amg", 1)
        once(False)
        m = once(False)
        G.grass_ctx_set_param(ctx, "lmax_amg", 0)
        # the same solve with PCG preconditioned by one V-cycle of the
        # sparsifier's multigrid (its hierarchy built inside the PCG phase)
        G.grass_ctx_set_param(ctx, "pcg_precond", 1)
        once(False)
        v = once(False)
        G.grass_ctx_set_param(ctx, "pcg_precond", 0)
        out = {"metric": "40M-unknown SDD solve s to 1e-3", "value": a["total"], "unit": "s",
               "higher_is_better": False,
               "workload": f"power-grid mesh {w['k']}x{w['k']} ({g.n} unknowns, {g.nnz} stored "
                           f"entries, {g.meta['vias']} vias, D ~ U[1e-4,1e-2]); r={w['r']}, "
                           f"t={w['t']}, sigma^2={w['sigma2']:g}, <= {w['rounds']} rounds, cap "
                           f"{w['cap_frac']:.0%} of n per round; FP32 embedding; PCG FP32 + FP64 "
                           f"residual to {w['tol']:g}",
               "phase_s": {"tree": a["tree"], "densify": a["densify"], "pcg": a["pcg"]},
               "pcg_iters": a["iters"], "rel_resid_fp64": a["rel"], "status": a["status"],
               "rounds": a["rounds"], "added": a["added"], "lmax_est": a["lmax"],
               "sparsifier_edges": a["n_s"],
               "e2e": {"value": e["total"], "unit": "s",
                       "h2d_bytes": sum(t.numel() * t.element_size() for t in hp),
                       "d2h_bytes": xh.numel() * 8},
               "lmax_capped": a["capped"], "stopped_similar": a["stopped"],
               "lmax_multigrid": {"value": m["total"], "unit": "s",
                                  "phase_s": {"tree": m["tree"], "densify": m["densify"],
                                              "pcg": m["pcg"]},
                                  "rounds": m["rounds"], "added": m["added"],
                                  "lmax_est": m["lmax"], "lmax_capped": m["capped"],
                                  "stopped_similar": m["stopped"], "pcg_iters": m["iters"],
                                  "rel_resid_fp64": m["rel"], "status": m["status"]},
               "pcg_multigrid": {"value": v["total"], "unit": "s",
                                 "phase_s": {"tree": v["tree"], "densify": v["densify"],
                                             "pcg": v["pcg"]},
                                 "pcg_iters": v["iters"], "rel_resid_fp64": v["rel"],
                                 "status": v["status"]},
               "host_generation_s": gen_s,
               "paper_context": "110 s, 34 PCG iterations: thupg8 (4.0e7 unknowns, 1.8e8 "
                                "nonzeros), one 2.67 GHz CPU core, Cholmod-factored sparsifier"}
    finally:
        G.grass_ctx_destroy(ctx)
    return out


# ---------------------------------------------------------------- serving

# one densification pass per request: with a 5 % cap the round-1 sparsifier is
# already sigma-similar on these meshes (estimated kappa ~ 20 <= 100), and a
# second allowed round would cost a full lambda_max estimate through inner CG
# only to confirm the stop
SERVE = dict(n_lo=1e4, n_hi=4.0e7, pool=12, seed=9, r=8, t=2, sigma2=100.0, rounds=1,
             lmax_iters=8, cap_frac=0.05, inner_tol=1e-2, inner_maxit=30, tol=1e-3,
             refine_tol=1e-3, pcg_inner_tol=1e-2, pcg_inner_maxit=1, maxit=5000,
             requests=1000, loads=(0.5, 0.8, 0.95), slots=4, capacity_requests=60)


def run_serve(G, args, w=SERVE) -> dict:
    """Serving: Poisson arrivals of sparsify+PCG requests on power-grid
    meshes whose sizes are log-uniform in [1e4, 4e7] unknowns (a pool of
    distinct meshes at log-spaced sizes; each request draws one and carries
    its own x), admitted by device-memory footprint on `slots` workers.
    Capacity = completions/s of a closed burst; then `requests` arrivals at
    each load fraction of it; latency = completion - submission."""
    import torch
    from synth import graphs, rng
    sides = sorted({int(round(np.sqrt(n))) for n in np.geomspace(w["n_lo"], w["n_hi"], w["pool"])})
    pool = []
    gen = torch.Generator().manual_seed(w["seed"])
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    for i, k in enumerate(sides):
        g = graphs.power_grid(k, w["seed"] + i)
        h0 = torch.randn(w["rounds"] * g.n * w["r"], generator=gen, dtype=torch.float64)
        v0 = torch.randn(w["rounds"] * g.n, generator=gen, dtype=torch.float64)
        pool.append(dict(g=g, rp=pin(g.rowptr), col=pin(g.col), val=pin(g.val),
                         h0=h0.pin_memory().numpy(), v0=v0.pin_memory().numpy(),
                         b=pin(rng.normal(w["seed"] + i, rng.STREAM_RHS, g.n))))
    P = lambda g: G.make_params(w["sigma2"], w["r"], w["t"], w["rounds"], w["lmax_iters"],
                                int(w["cap_frac"] * g.n), G.GRASS_FP32, w["inner_tol"],
                                w["inner_maxit"])
    rs = np.random.default_rng(w["seed"])
    srv = G.Server(0, w["slots"], 0)
    grid_sms = getattr(args, "serve_grid_sms", 0) or 0
    srv.set_param("grid_sms", grid_sms)
    n_req = getattr(args, "serve_requests", None) or w["requests"]

    def submit(j):
        e = pool[j]
        x = np.empty(e["g"].n)
        t = srv.submit(e["rp"], e["col"], e["val"], e["h0"], e["v0"], e["b"], x, P(e["g"]),
                       w["tol"], w["maxit"], G.GRASS_FP32, w["refine_tol"], w["pcg_inner_tol"],
                       w["pcg_inner_maxit"])
        return t

    def collect(tickets, picks):
        res = [srv.wait(t) for t in tickets]
        bad = [r.error.decode() for r in res if r.status != 0]
        lat = np.array([1e3 * (r.t_done - r.t_submit) for r in res])
        span = max(r.t_done for r in res) - min(r.t_submit for r in res)
        return res, bad, lat, span

    try:
        # warm every pool size once, then the closed burst for capacity
        collect([submit(j) for j in range(len(pool))], None)
        picks = rs.integers(0, len(pool), w["capacity_requests"])
        res, bad, lat, span = collect([submit(int(j)) for j in picks], picks)
        capacity = len(res) / span
        loads = []
        for f in (w["loads"] if not getattr(args, "serve_capacity_only", False) else ()):
            rate = f * capacity
            picks = rs.integers(0, len(pool), n_req)
            gaps = rs.exponential(1.0 / rate, n_req)
            t0 = time.perf_counter()
            due = t0 + np.cumsum(gaps)
            tickets = []
            for j, d in zip(picks, due):
                dt = d - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                tickets.append(submit(int(j)))
            res, bad2, lat, span = collect(tickets, picks)
            bad += bad2
            loads.append({"load": f, "rate_rps": rate, "requests": len(res),
                          "p50_ms": float(np.percentile(lat, 50)),
                          "p99_ms": float(np.percentile(lat, 99)),
                          "throughput_rps": len(res) / span,
                          "max_in_flight": max(r.in_flight_at_admit for r in res),
                          "mean_queue_ms": float(np.mean([1e3 * (r.t_admit - r.t_submit) for r in res])),
                          "pcg_iters_max": max(r.solve.iters for r in res),
                          "rel_resid_max": max(r.solve.rel_resid_fp64 for r in res)})
        st = srv.stats()
    finally:
        srv.close()
    if not loads:
        return {"metric": "serve capacity", "value": capacity, "unit": "requests/s",
                "higher_is_better": True, "grid_sms": grid_sms, "slots": w["slots"],
                "n_errors": len(bad), "errors": bad[:5],
                "capacity_latency_ms": {"p50": float(np.percentile(lat, 50)),
                                        "max": float(lat.max())}}
    mid = loads[len(loads) // 2]
    return {"metric": "serve p50/p99 latency", "value": mid["p99_ms"], "unit": "ms (p99)",
            "higher_is_better": False, "p50_ms": mid["p50_ms"], "load_of_value": mid["load"],
            "capacity_rps": capacity, "loads": loads, "errors": bad[:5], "n_errors": len(bad),
            "slots": w["slots"], "max_running": st["max_running"], "grid_sms": grid_sms,
            "requests_per_load": n_req,
            "pool_sizes": [p["g"].n for p in pool],
            "workload": "Poisson stream of sparsify+PCG requests, power-grid meshes (U[0.1,10] "
                        "wires, 1% vias of weight 100, pads U[1e-4,1e-2]), sizes log-uniform in "
                        f"[{w['n_lo']:.0e}, {w['n_hi']:.0e}] unknowns; r={w['r']}, t={w['t']}, "
                        f"sigma^2={w['sigma2']:g}, <= {w['rounds']} rounds, PCG to {w['tol']:g}"}


# ---------------------------------------------------------------- batching

BATCH = dict(count=256, seed=7, r=8, t=2, sigma2=100.0, lmax_iters=8, tol=1e-3, maxit=5000,
             inner=1, reps=3)


def run_batch(G, w=BATCH) -> dict:
    """256 graphs of uneven size (2D grids 32^2..512^2, rings of 1e3..2e5
    nodes with n/4 chords, w ~ U[1,10), D = 1e-3 I) as one block-diagonal
    batch: forest, autotuned forest-solve shape, one densification round
    (r=8, t=2, sigma^2=100, FP32 embedding) and PCG of every graph to 1e-3
    (FP32 vectors, FP64 scalars), the outer iteration replayed as a CUDA
    graph.  Compared with the plain FP64 single-graph method run on each
    graph in turn at the same 1e-3 accuracy."""
    import torch
    from synth import graphs
    t0 = time.perf_counter()
    gs = graphs.config_batch(w["count"], w["seed"])
    u, off = graphs.batch_union(gs)
    gen = torch.Generator().manual_seed(w["seed"])
    h0 = torch.randn(u.n * w["r"], generator=gen, dtype=torch.float64)
    v0 = torch.randn(u.n, generator=gen, dtype=torch.float64)
    b = torch.randn(u.n, generator=gen, dtype=torch.float64)
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(stream):
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        rp, col, val = d(u.rowptr), d(u.col), d(u.val)
        h0d, v0d, bd = h0.cuda(), v0.cuda(), b.cuda()
        x = torch.zeros(u.n, dtype=torch.float64, device="cuda")
        ctx = G.grass_ctx_create(stream)
        P = G.make_params(w["sigma2"], w["r"], w["t"], 1, w["lmax_iters"], 0, G.GRASS_FP32,
                          1e-2, 30)
        nseg = len(gs)
        try:
            tree = G.grass_build_forest(ctx, rp, col, val, off)
            best, best_ms = G.grass_autotune(ctx, tree, w["r"], G.GRASS_FP32)
            row_best, row_ms = G.grass_autotune_rows(ctx, tree, w["r"], G.GRASS_FP32)
            G.grass_tree_destroy(tree)

            def one(prec):
                stream.synchronize()
                t0 = time.perf_counter()
                tr = G.grass_build_forest(ctx, rp, col, val, off)
                t1 = time.perf_counter()
                S, st, rows = G.grass_densify_batch(ctx, tr, P, h0d, v0d, nseg)
                t2 = time.perf_counter()
                s, ps, its, res = G.grass_pcg_solve_batch(ctx, S, bd, x, w["tol"], w["maxit"],
                                                          prec, w["inner"], nseg)
                stream.synchronize()
                t3 = time.perf_counter()
                G.grass_sparsifier_destroy(S)
                G.grass_tree_destroy(tr)
                return dict(total=t3 - t0, forest=t1 - t0, densify=t2 - t1, pcg=t3 - t2, status=s,
                            iters_max=max(its), iters_median=float(np.median(its)),
                            rel_max=max(res), embedded=st.offtree_embedded, added=st.added,
                            stopped=sum(1 for r_ in rows if np.isinf(r_[2])))

            one(G.GRASS_FP32)
            l0 = G.grass_launch_count(ctx)
            runs = [one(G.GRASS_FP32) for _ in range(w["reps"])]
            launches = (G.grass_launch_count(ctx) - l0) // w["reps"]
            best_run = min(runs, key=lambda r_: r_["total"])
            f64 = one(G.GRASS_FP64)
        finally:
            G.grass_ctx_destroy(ctx)
        # the plain FP64 method, one graph after another, same accuracy
        ctx1 = G.grass_ctx_create(stream)
        Pp = G.make_params(w["sigma2"], w["r"], w["t"], 1, w["lmax_iters"], 0, G.GRASS_FP64,
                           1e-10, 1000)
        seq_worst = 0.0
        try:
            def seq():
                nonlocal seq_worst
                stream.synchronize()
                t0 = time.perf_counter()
                for k, g in enumerate(gs):
                    sl = slice(off[k], off[k + 1])
                    tr = G.grass_build_tree(ctx1, rp_k[k], col_k[k], val_k[k], 0)
                    S, st = G.grass_densify(ctx1, tr, Pp, h0d[off[k] * w["r"]:off[k + 1] * w["r"]],
                                            v0d[sl])
                    xs = x[sl]
                    s, ps = G.grass_pcg_solve(ctx1, S, bd[sl], xs, w["tol"], w["maxit"],
                                              G.GRASS_FP64, 1e-2, 1e-6, 1)
                    seq_worst = max(seq_worst, ps.rel_resid_fp64)
                    G.grass_sparsifier_destroy(S)
                    G.grass_tree_destroy(tr)
                stream.synchronize()
                return time.perf_counter() - t0
            rp_k, col_k, val_k = [], [], []
            for g in gs:
                rp_k.append(d(g.rowptr))
                col_k.append(d(g.col))
                val_k.append(d(g.val))
            seq()
            seq_s = seq()
        finally:
            G.grass_ctx_destroy(ctx1)
    n_edges = int(sum(g.m for g in gs))
    out = {"metric": "batch of 256 graphs sparsified and solved to 1e-3", "value": best_run["total"],
           "unit": "s", "higher_is_better": False, "graphs_per_s": nseg / best_run["total"],
           "offtree_edges_embedded_per_s": best_run["embedded"] / best_run["densify"],
           "phase_s": {k: best_run[k] for k in ("forest", "densify", "pcg")},
           "pcg_iters_max": best_run["iters_max"], "pcg_iters_median": best_run["iters_median"],
           "rel_resid_max": best_run["rel_max"], "status": best_run["status"],
           "graphs_already_similar": best_run["stopped"], "edges_added": best_run["added"],
           "gpu_launches_per_batch": launches,
           "batched_fp64_vectors_s": f64["total"],
           "sequential_plain_fp64_s": seq_s, "sequential_rel_resid_max": seq_worst,
           "speedup_vs_sequential_fp64": seq_s / best_run["total"],
           "autotune": {"tree_threads": best[0], "tree_blocks_per_sm": best[1],
                        "tree_tail_items": best[2], "forest_solve_ms_r8": best_ms,
                        "spmm_chunk_cap": row_best[0], "spmm_variant": row_best[1],
                        "heat_form": row_best[2], "spmm_ms_r8": row_ms[0],
                        "heat_ms_r8": row_ms[1]},
           "workload": f"{nseg} graphs ({u.n} nodes, {n_edges} edges): 2D grids side "
                       "log-uniform in [32,512] and rings of log-uniform [1e3,2e5] nodes with n/4 "
                       "chords, w ~ U[1,10), D = 1e-3 I; r=8, t=2, sigma^2=100, one round; PCG to "
                       "1e-3 (FP32 vectors, FP64 scalars, forest solve + 1 inner CG step)",
           "host_generation_s": gen_s}
    return out


# ---------------------------------------------------------------- extras (outside the timed region)

def round_bytes(n: int, m: int, nnz: int, moff: int, r: int, t: int, s: int) -> float:
    """Algorithmic bytes of one embedding round by the formulas of the scope
    table (each array once, perfect reuse of gathered rows): t (SpMM + tree
    solve) + heat, SpMM = 8(n+1) + nnz(4+s) + 2nrs, tree = 2n(4+2s) + 6nrs,
    heat = moff(8+s) + nrs + moff s."""
    spmm = 8 * (n + 1) + nnz * (4 + s) + 2 * n * r * s
    tree = 2 * n * (4 + 2 * s) + 6 * n * r * s
    heat = moff * (8 + s) + n * r * s + moff * s
    return t * (spmm + tree) + heat


def per_round(st: dict, g, w: dict, peak: float) -> list:
    """Off-tree edges embedded per second of each round's embedding (power
    steps + heat, host wall time of a call that ends synchronised), and for
    round 1 (tree solves, no inner CG) its fraction of the HBM roofline."""
    s = 4 if w["embed"] == "fp32" else 8
    out = []
    for k in range(st["rounds"]):
        ms = st["ms_embed_round"][k]
        moff = st["embedded_round"][k]
        row = {"round": k + 1, "offtree_edges": moff, "ms": ms,
               "edges_per_s": moff / (ms / 1e3) if ms > 0 else None}
        if k == 0:
            by = round_bytes(g.n, g.m, g.nnz, moff, w["r"], w["t"], s)
            row.update(algorithmic_bytes=by, GBps=by / (ms / 1e3) / 1e9,
                       frac_of_measured_hbm=by / (ms / 1e3) / 1e9 / peak)
        else:
            row["note"] = "sparsifier solves by inner CG (t x inner iterations tree solves)"
        out.append(row)
    return out


def c2_extras(G, ctx, w: dict, g, rp, col, val, h0d, v0d, bd, P, peak: float,
              pcg_mg: bool = True) -> dict:
    """On the step's sparsifier: the lambda estimates with tight inner solves
    (certifying the stop decision), the plain FP64 method at the same 1e-8
    accuracy, and the PCG iteration count and time for inner budgets 0 (tree
    preconditioner) .. 8 (one-step FP32 PCG passes, FP64 refinement)."""
    import torch
    out = {}
    tree = G.grass_build_tree(ctx, rp, col, val, 0)
    S, st = G.grass_densify(ctx, tree, P, h0d, v0d)
    try:
        d = st.as_dict()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lmin = G.grass_lambda_min(ctx, S)
        vk = torch.randn(g.n, dtype=torch.float64, device="cuda",
                         generator=torch.Generator(device="cuda").manual_seed(11))
        lmax = G.grass_lambda_max(ctx, S, vk, 30, G.GRASS_FP64, 1e-10, 3000)
        out["kappa_check"] = {
            "lambda_min_est": lmin, "lambda_max_tight": lmax, "kappa_tight": lmax / lmin,
            "sigma2": w["sigma2"], "bench_lambda_max_est": d["lmax_est"][-1],
            "bench_stopped_similar": d["stopped_similar"],
            "method": "30 generalized power steps from a fresh vector, FP64, inner CG to "
                      "1e-10 (Rayleigh quotient: a lower bound of the true lambda_max)",
            "s": time.perf_counter() - t0}
        sweep = []
        x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
        # the tree solve with 0-8 inner steps on the sparsifier, then the V-cycle
        G.grass_ctx_set_param(ctx, "pcg_precond", 0)
        for inner in (0, 1, 2, 4, 8):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            stt, ps = G.grass_pcg_solve(ctx, S, bd, x, w["pcg_tol"], w["pcg_maxit"], G.GRASS_FP32,
                                        w["refine_tol"], w["pcg_inner_tol"], inner)
            torch.cuda.synchronize()
            sweep.append({"inner_maxit": inner, "iters": ps.iters, "ms": 1e3 * (time.perf_counter() - t0),
                          "rel_resid_fp64": ps.rel_resid_fp64, "status": stt})
        # the sparsifier's multigrid V-cycle as the preconditioner (setup included)
        G.grass_ctx_set_param(ctx, "pcg_precond", 1)
        for prec_name, pp in (("fp32", G.GRASS_FP32), ("fp64", G.GRASS_FP64)):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            stt, ps = G.grass_pcg_solve(ctx, S, bd, x, w["pcg_tol"], w["pcg_maxit"], pp,
                                        w["refine_tol"], w["pcg_inner_tol"], 0)
            torch.cuda.synchronize()
            sweep.append({"preconditioner": f"multigrid V-cycle of L_S + D ({prec_name}; first "
                          "call includes the hierarchy setup)" if prec_name == "fp32" else
                          "multigrid V-cycle of L_S + D (fp64)", "iters": ps.iters,
                          "ms": 1e3 * (time.perf_counter() - t0),
                          "rel_resid_fp64": ps.rel_resid_fp64, "status": stt})
        G.grass_ctx_set_param(ctx, "pcg_precond", 1 if pcg_mg else 0)
        out["pcg_inner_sweep"] = sweep
        # lambda_max of the final sparsifier by multigrid-CG solves (8 steps, 1e-6)
        G.grass_ctx_set_param(ctx, "lmax_amg", 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lm_amg = G.grass_lambda_max(ctx, S, vk, 8, G.GRASS_FP64, 1e-6, 500)
        torch.cuda.synchronize()
        out["kappa_check"]["lambda_max_amg_8_steps"] = lm_amg
        out["kappa_check"]["lambda_max_amg_s"] = time.perf_counter() - t0
        G.grass_ctx_set_param(ctx, "lmax_amg", 0)
    finally:
        G.grass_sparsifier_destroy(S)
        G.grass_tree_destroy(tree)
    # the plain FP64 method: FP64 embedding and FP64 PCG to the same tolerance
    P64 = G.make_params(w["sigma2"], w["r"], w["t"], w["rounds"], w["lmax_iters"],
                        int(w["cap_frac"] * g.n), G.GRASS_FP64, w["inner_tol"], w["inner_maxit"])
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")

    def fp64_step():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tr = G.grass_build_tree(ctx, rp, col, val, 0)
        t1 = time.perf_counter()
        S2, st2 = G.grass_densify(ctx, tr, P64, h0d, v0d)
        t2 = time.perf_counter()
        x.zero_()
        s2, ps2 = G.grass_pcg_solve(ctx, S2, bd, x, w["pcg_tol"], w["pcg_maxit"], G.GRASS_FP64,
                                    w["refine_tol"], w["pcg_inner_tol"], w["pcg_inner_maxit"])
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        G.grass_sparsifier_destroy(S2)
        G.grass_tree_destroy(tr)
        return {"ms_per_step": 1e3 * (t3 - t0),
                "phase_ms": {"tree": 1e3 * (t1 - t0), "densify": 1e3 * (t2 - t1), "pcg": 1e3 * (t3 - t2)},
                "edges_embedded": st2.offtree_embedded, "rounds": st2.rounds, "added": st2.added,
                "pcg_iters": ps2.iters, "rel_resid_fp64": ps2.rel_resid_fp64, "status": s2}
    fp64_step()
    out["fp64_path"] = fp64_step()
    out["fp64_path"]["edges_per_s"] = out["fp64_path"]["edges_embedded"] / (
        out["fp64_path"]["ms_per_step"] / 1e3)
    return out


def c1_latency(G, reps: int = 10) -> dict:
    """The 64 x 64 grid, plain FP64 method (tree, one round r=8 t=2
    sigma^2=100, PCG to 1e-3): latency of the whole path from the device CSR."""
    import torch
    w = WORKLOADS["grid2d_64"]
    g, h0, v0, b = make_inputs(w)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, col, val, h0d, v0d, bd = d(g.rowptr), d(g.col), d(g.val), d(h0), d(v0), d(b)
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    ctx = G.grass_ctx_create()
    P = G.make_params(w["sigma2"], w["r"], w["t"], w["rounds"], w["lmax_iters"], 0, G.GRASS_FP64,
                      w["inner_tol"], w["inner_maxit"])
    times, last = [], None
    try:
        for k in range(reps + 3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tree = G.grass_build_tree(ctx, rp, col, val, 0)
            S, st = G.grass_densify(ctx, tree, P, h0d, v0d)
            x.zero_()
            s, ps = G.grass_pcg_solve(ctx, S, bd, x, w["pcg_tol"], w["pcg_maxit"], G.GRASS_FP64,
                                      w["refine_tol"], w["pcg_inner_tol"], w["pcg_inner_maxit"])
            torch.cuda.synchronize()
            if k >= 3:
                times.append(1e6 * (time.perf_counter() - t0))
            last = (st, ps)
            G.grass_sparsifier_destroy(S)
            G.grass_tree_destroy(tree)
    finally:
        G.grass_ctx_destroy(ctx)
    st, ps = last
    return {"workload": describe(w, g), "latency_us_median": float(np.median(times)),
            "latency_us_min": float(np.min(times)), "reps": reps, "added": st.added,
            "pcg_iters": ps.iters, "rel_resid_fp64": ps.rel_resid_fp64,
            "edges_embedded_per_s": st.offtree_embedded / (np.median(times) / 1e6)}


C3 = dict(n=4_000_000, seed=3, r=24, t=3, sigma2=500.0, rounds=3, lmax_iters=8, cap_frac=0.02,
          embed="fp32", inner_tol=1e-2, inner_maxit=30)


def c3_powerlaw(G, peak: float, w=C3) -> dict:
    """Chung-Lu power-law graph (4M sampled nodes, mean degree 10, exponent
    2.1, unit weights, largest component), r=24, t=3, sigma^2=500, FP32
    embedding, <= 3 densification rounds with a 2 % per-round cap: spanning
    tree + densification from the device CSR (one warm run, one timed)."""
    import torch
    from synth import graphs, rng
    t0 = time.perf_counter()
    g = graphs.chung_lu(w["n"], w["seed"])
    gen_s = time.perf_counter() - t0
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, col, val = d(g.rowptr), d(g.col), d(g.val)
    gen = torch.Generator(device="cuda").manual_seed(w["seed"])
    h0 = torch.randn(w["rounds"] * g.n * w["r"], generator=gen, device="cuda", dtype=torch.float64)
    v0 = torch.randn(w["rounds"] * g.n, generator=gen, device="cuda", dtype=torch.float64)
    P = G.make_params(w["sigma2"], w["r"], w["t"], w["rounds"], w["lmax_iters"],
                      int(w["cap_frac"] * g.n), G.GRASS_FP32, w["inner_tol"], w["inner_maxit"])
    ctx = G.grass_ctx_create()
    try:
        def run():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tree = G.grass_build_tree(ctx, rp, col, val, 0)
            t1 = time.perf_counter()
            S, st = G.grass_densify(ctx, tree, P, h0, v0)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            n_s, _ = G.grass_sparsifier_info(S)
            rounds = G.grass_tree_info(tree)[2]
            G.grass_sparsifier_destroy(S)
            G.grass_tree_destroy(tree)
            return st.as_dict(), 1e3 * (t1 - t0), 1e3 * (t2 - t1), n_s, rounds
        run()
        st, tree_ms, dens_ms, n_s, frounds = run()
    finally:
        G.grass_ctx_destroy(ctx)
    deg = np.diff(g.rowptr) - 1
    wdesc = dict(embed="fp32", r=w["r"], t=w["t"])
    return {"workload": f"Chung-Lu power law ({w['n']} sampled nodes, LCC {g.n} nodes, {g.m} edges, "
                        f"max degree {int(deg.max())}, unit weights); r={w['r']}, t={w['t']}, "
                        f"sigma^2={w['sigma2']:g}, <= {w['rounds']} rounds, cap 2 % of n; FP32",
            "n": g.n, "m": g.m, "tree_ms": tree_ms, "densify_ms": dens_ms,
            "edges_embedded": st["offtree_embedded"],
            "edges_embedded_per_s": st["offtree_embedded"] / ((tree_ms + dens_ms) / 1e3),
            "per_round": per_round(st, g, wdesc, peak), "densify": st,
            "sparsifier_edges": n_s, "tree_factor_rounds": frounds, "host_generation_s": gen_s}


def partition_mesh(G, side: int = 1000, seed: int = 12, iters: int = 5) -> dict:
    """Spectral partitioning (Sec. V-F, Table VI's mesh_1M stand-in): a
    side x side 2D mesh with weights U[1,10) and no diagonal load; the
    sparsifier (r=8, t=2, sigma^2=200, <= 3 rounds, cap 5 % of n, FP32), then
    `iters` inverse power iterations with PCG preconditioned by it to 1e-3
    (FP32 + FP64 refinement) and the sign cut; the reference cut uses FP64
    solves to 1e-10.  T_I excludes the sparsification, as in the paper."""
    import torch
    from synth import graphs, rng
    g = graphs.grid2d_uniform(side, side, seed, D=0.0)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, col, val = d(g.rowptr), d(g.col), d(g.val)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    h0 = torch.randn(3 * g.n * 8, generator=gen, device="cuda", dtype=torch.float64)
    v0 = torch.randn(3 * g.n, generator=gen, device="cuda", dtype=torch.float64)
    x0 = torch.randn(g.n, generator=gen, device="cuda", dtype=torch.float64)
    P = G.make_params(200.0, 8, 2, 3, 8, int(0.05 * g.n), G.GRASS_FP32, 1e-2, 30)
    ctx = G.grass_ctx_create()
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tree = G.grass_build_tree(ctx, rp, col, val, 0)
        S, st = G.grass_densify(ctx, tree, P, h0, v0)
        torch.cuda.synchronize()
        t_sp = time.perf_counter() - t0
        s_fast = torch.empty(g.n, dtype=torch.uint8, device="cuda")
        s_ref = torch.empty_like(s_fast)
        # tree-preconditioned solves for comparison (capped at 2000 iterations each)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st_tree, f_tree = G.grass_fiedler(ctx, S, x0, iters, 1e-3, 2000 * iters, G.GRASS_FP32, 0,
                                          None, s_fast)
        torch.cuda.synchronize()
        t_tree = time.perf_counter() - t0
        # the sparsifier's multigrid V-cycle preconditions every solve
        G.grass_ctx_set_param(ctx, "pcg_precond", 1)
        G.grass_fiedler(ctx, S, x0, iters, 1e-3, 50000, G.GRASS_FP32, 1, None, s_fast)   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sf, ff = G.grass_fiedler(ctx, S, x0, iters, 1e-3, 50000, G.GRASS_FP32, 1, None, s_fast)
        torch.cuda.synchronize()
        t_i = time.perf_counter() - t0
        sr, fr = G.grass_fiedler(ctx, S, x0, iters, 1e-10, 100000, G.GRASS_FP64, 0, None, s_ref)
        rel_err = float((s_fast != s_ref).float().mean().item())
        n_s, _ = G.grass_sparsifier_info(S)
        G.grass_sparsifier_destroy(S)
        G.grass_tree_destroy(tree)
    finally:
        G.grass_ctx_destroy(ctx)
    return {"workload": f"{side}x{side} 2D mesh, w ~ U[1,10), D = 0; sparsifier r=8 t=2 "
                        f"sigma^2=200 <= 3 rounds cap 5 %; {iters} inverse power iterations, PCG "
                        "to 1e-3 (FP32 + FP64 refinement) preconditioned by the sparsifier",
            "n": g.n, "T_I_s": t_i, "sparsify_s": t_sp, "pcg_iters": ff.pcg_iters,
            "all_solves_converged": sf == 0, "worst_rel_resid": ff.worst_rel_resid,
            "v_pos_over_v_neg": ff.n_pos / max(ff.n_neg, 1), "rel_err_vs_fp64_1e-10": rel_err,
            "rayleigh": ff.rayleigh, "reference_pcg_iters": fr.pcg_iters,
            "preconditioner": "multigrid V-cycle of the sparsifier (reference: the same, FP64)",
            "tree_preconditioned": {"T_I_s": t_tree, "pcg_iters": f_tree.pcg_iters,
                                    "converged": st_tree == 0,
                                    "worst_rel_resid": f_tree.worst_rel_resid},
            "sparsifier_edges": n_s, "densify_rounds": st.rounds,
            "paper_context": "Table VI mesh_1M: |V+|/|V-| 1.01, T_I 1.7 s (one CPU core), "
                             "Rel.Err 3.3e-3 vs the direct solver"}


def hair_comb(G, k: int = 200, add: int = 400) -> dict:
    """The hair-comb spanning tree of the k x k unit mesh (a caller's tree):
    lambda_max estimate of the tree (eight power steps), then one random
    vector, one power step, the `add` hottest off-tree edges added, and the
    estimate again (30 steps, inner CG to 1e-10)."""
    import torch
    from synth import graphs, rng
    g = graphs.grid((k, k), None, 0.0)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, col, val = d(g.rowptr), d(g.col), d(g.val)
    u, v = graphs.hair_comb_edges(k, k)
    ctx = G.grass_ctx_create()
    tree = S = None
    try:
        eu = torch.empty(g.m, dtype=torch.int32, device="cuda")
        ev = torch.empty_like(eu)
        t0 = G.grass_build_tree(ctx, rp, col, val, 0)          # for its edge list only
        G.grass_tree_graph(ctx, t0, eu, ev, None, None)
        G.grass_tree_destroy(t0)
        key = eu.cpu().numpy().astype(np.int64) * g.n + ev.cpu().numpy()
        ids = np.searchsorted(key, u * g.n + v).astype(np.int64)
        tree = G.grass_tree_from_edges(ctx, rp, col, val, d(ids), 0)
        S = G.grass_sparsifier_create(ctx, tree)
        v0 = d(rng.normal(3, rng.STREAM_V0, g.n))
        before = G.grass_lambda_max(ctx, S, v0, 8, G.GRASS_FP64, 1e-12, 100)
        _, moff = G.grass_sparsifier_info(S)
        heat = torch.empty(moff, dtype=torch.float64, device="cuda")
        G.grass_embed(ctx, S, d(rng.gaussian_block(3, rng.STREAM_H0, g.n, 1)), 1, 1, G.GRASS_FP64,
                      1e-12, 100, None, heat)
        acc = torch.empty(moff, dtype=torch.int64, device="cuda")
        na, _ = G.grass_filter(ctx, S, heat, G.GRASS_FP64, 1e-30, 1.0, 1.0, 1, add, acc)
        G.grass_sparsifier_add(ctx, S, acc[:na].contiguous())
        after = G.grass_lambda_max(ctx, S, v0, 30, G.GRASS_FP64, 1e-10, 3000)
    finally:
        if S:
            G.grass_sparsifier_destroy(S)
        if tree:
            G.grass_tree_destroy(tree)
        G.grass_ctx_destroy(ctx)
    return {"workload": f"{k}x{k} unit mesh, hair-comb spanning tree (spine y=0, one tooth per "
                        f"column); t=1, one random vector, top {add} by heat added",
            "lambda_max_tree": before, "lambda_max_after": after, "added": na,
            "paper_context": "Sec. V-C: about 64,000 for the tree, about 100 after adding the top "
                             "400 edges (figure not reproduced by this reading; see DESIGN)"}


def densify_budget(G, w: dict, g, rp, col, val, bd, rounds=(3, 6, 16)) -> dict:
    """The 100^3 step's densification with more rounds at the same per-round
    cap, lambda_max by the step's tree-preconditioned inner CG and by
    multigrid-CG solves: sparsifier edges, the lambda_max estimates, the
    edges each round added, and the PCG iterations and time with the
    sparsifier applied as in the step (one inner step) and by its multigrid
    V-cycle.  The paper's 36-40 iterations at sigma^2 = 200 (Table V) need a
    sparsifier whose kappa reaches sigma^2; this shows how the count moves
    with the densification budget."""
    import torch
    from synth import rng
    ctx = G.grass_ctx_create(torch.cuda.current_stream())
    out = {"rounds_cap": f"{w['cap_frac']:.0%} of n per round", "runs": []}
    pcg_prec = G.GRASS_FP32 if w["pcg"] == "fp32" else G.GRASS_FP64
    try:
        for amg in (0, 1):
            G.grass_ctx_set_param(ctx, "lmax_amg", amg)
            for R in rounds:
                h0 = torch.from_numpy(np.concatenate(
                    [rng.gaussian_block(w["seed"], rng.STREAM_H0 + k, g.n, w["r"])
                     for k in range(R)])).cuda()
                v0 = torch.from_numpy(np.concatenate(
                    [rng.normal(w["seed"], rng.STREAM_V0 + k, g.n) for k in range(R)])).cuda()
                P = G.make_params(w["sigma2"], w["r"], w["t"], R, w["lmax_iters"],
                                  int(w["cap_frac"] * g.n),
                                  G.GRASS_FP32 if w["embed"] == "fp32" else G.GRASS_FP64,
                                  w["inner_tol"], w["inner_maxit"])
                tree = G.grass_build_tree(ctx, rp, col, val, 0)
                S = None
                try:
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    S, st = G.grass_densify(ctx, tree, P, h0, v0)
                    torch.cuda.synchronize()
                    dd = st.as_dict()
                    r_ = {"lambda_max": "multigrid-CG" if amg else "tree-CG (the step's)",
                          "rounds_max": R, "rounds": dd["rounds"],
                          "densify_ms": 1e3 * (time.perf_counter() - t0),
                          "sparsifier_edges": G.grass_sparsifier_info(S)[0],
                          "lmax_est": dd["lmax_est"], "lmax_capped": dd["lmax_capped"],
                          "added_round": dd["added_round"],
                          "stopped_similar": dd["stopped_similar"]}
                    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
                    for name, pre, inner in (("pcg_one_inner_step", 0, w["pcg_inner_maxit"]),
                                             ("pcg_multigrid", 1, 0)):
                        G.grass_ctx_set_param(ctx, "pcg_precond", pre)
                        if pre:
                            x.zero_()
                            G.grass_pcg_solve(ctx, S, bd, x, w["pcg_tol"], w["pcg_maxit"],
                                              pcg_prec, w["refine_tol"], w["pcg_inner_tol"],
                                              inner)
                        x.zero_()
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        s_, ps = G.grass_pcg_solve(ctx, S, bd, x, w["pcg_tol"], w["pcg_maxit"],
                                                   pcg_prec, w["refine_tol"], w["pcg_inner_tol"],
                                                   inner)
                        torch.cuda.synchronize()
                        r_[name] = {"iters": ps.iters,
                                    "ms": 1e3 * (time.perf_counter() - t0), "status": s_}
                    G.grass_ctx_set_param(ctx, "pcg_precond", 0)
                    out["runs"].append(r_)
                finally:
                    if S:
                        G.grass_sparsifier_destroy(S)
                    G.grass_tree_destroy(tree)
    finally:
        G.grass_ctx_destroy(ctx)
    return out


def lsst_vs_mst(G, w: dict, P, g=None, h0d=None, v0d=None, bd=None, label: str = "") -> dict:
    """The maximum-weight tree against the low-stretch tree (Sec. III-B) on
    one workload: construction time, total stretch st_T(G), PCG with the
    tree alone as preconditioner, and the densified sparsifier (rounds,
    edges, lambda_max estimates) with its PCG, both under the step's
    parameters."""
    import torch
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, col, val = d(g.rowptr), d(g.col), d(g.val)
    pcg_prec = G.GRASS_FP32 if w["pcg"] == "fp32" else G.GRASS_FP64
    out = {"workload": label}
    ctx = G.grass_ctx_create(torch.cuda.current_stream())
    try:
        for kind in ("mst", "lsst"):
            r_ = {}
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if kind == "mst":
                tree = G.grass_build_tree(ctx, rp, col, val, 0)
            else:
                tree, ls = G.grass_build_lsst(ctx, rp, col, val, 1, 0)
                r_["construction"] = ls
            torch.cuda.synchronize()
            r_["build_ms"] = 1e3 * (time.perf_counter() - t0)
            S = None
            try:
                t0 = time.perf_counter()
                r_["total_stretch"] = G.grass_tree_stretch(ctx, tree)
                r_["stretch_ms"] = 1e3 * (time.perf_counter() - t0)
                r_["mean_stretch"] = r_["total_stretch"] / g.m
                S = G.grass_sparsifier_create(ctx, tree)
                x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
                t0 = time.perf_counter()
                st_, ps = G.grass_pcg_solve(ctx, S, bd, x, w["pcg_tol"], w["pcg_maxit"], pcg_prec,
                                            w["refine_tol"], w["pcg_inner_tol"], 0)
                r_["pcg_tree_only"] = {"iters": ps.iters, "ms": 1e3 * (time.perf_counter() - t0),
                                       "rel_resid_fp64": ps.rel_resid_fp64, "status": st_}
                G.grass_sparsifier_destroy(S)
                S = None
                if h0d is not None:
                    t0 = time.perf_counter()
                    S, dst = G.grass_densify(ctx, tree, P, h0d, v0d)
                    dd = dst.as_dict()
                    r_["densify"] = {"ms": 1e3 * (time.perf_counter() - t0), "rounds": dd["rounds"],
                                     "added": dd["added"], "lmax_est": dd["lmax_est"],
                                     "lmax_capped": dd.get("lmax_capped"),
                                     "stopped_similar": dd["stopped_similar"]}
                    x.zero_()
                    t0 = time.perf_counter()
                    st_, ps = G.grass_pcg_solve(ctx, S, bd, x, w["pcg_tol"], w["pcg_maxit"],
                                                pcg_prec, w["refine_tol"], w["pcg_inner_tol"],
                                                w["pcg_inner_maxit"])
                    r_["pcg_sparsifier"] = {"iters": ps.iters,
                                            "ms": 1e3 * (time.perf_counter() - t0),
                                            "rel_resid_fp64": ps.rel_resid_fp64, "status": st_}
                    # the same sparsifier applied by its multigrid V-cycle
                    # (pcg_precond = 1; the first call builds the hierarchy)
                    G.grass_ctx_set_param(ctx, "pcg_precond", 1)
                    try:
                        x.zero_()
                        G.grass_pcg_solve(ctx, S, bd, x, w["pcg_tol"], w["pcg_maxit"], pcg_prec,
                                          w["refine_tol"], w["pcg_inner_tol"], 0)
                        x.zero_()
                        t0 = time.perf_counter()
                        st_, ps = G.grass_pcg_solve(ctx, S, bd, x, w["pcg_tol"], w["pcg_maxit"],
                                                    pcg_prec, w["refine_tol"], w["pcg_inner_tol"], 0)
                        r_["pcg_sparsifier_multigrid"] = {
                            "iters": ps.iters, "ms": 1e3 * (time.perf_counter() - t0),
                            "rel_resid_fp64": ps.rel_resid_fp64, "status": st_}
                    finally:
                        G.grass_ctx_set_param(ctx, "pcg_precond", 0)
            finally:
                if S:
                    G.grass_sparsifier_destroy(S)
                G.grass_tree_destroy(tree)
            out[kind] = r_
    finally:
        G.grass_ctx_destroy(ctx)
    return out


def lsst_extras(G, w: dict, P, g, h0d, v0d, bd) -> dict:
    """lsst_vs_mst on the step's workload (with densification) and on a
    1000 x 1000 unit mesh with D = 1e-3 I (tree-only PCG to 1e-3)."""
    import torch
    from synth import graphs, rng
    res = {"grid3d": lsst_vs_mst(G, w, P, g, h0d, v0d, bd, describe(w, g))}
    gm = graphs.grid((1000, 1000), None, 1e-3)
    wm = dict(w, pcg_tol=1e-3, pcg="fp32")
    bm = torch.from_numpy(rng.normal(4, rng.STREAM_RHS, gm.n)).cuda()
    R = w["rounds"]
    hm = torch.from_numpy(np.concatenate([rng.gaussian_block(4, rng.STREAM_H0 + k, gm.n, w["r"])
                                          for k in range(R)])).cuda()
    vm = torch.from_numpy(np.concatenate([rng.normal(4, rng.STREAM_V0 + k, gm.n)
                                          for k in range(R)])).cuda()
    Pm = G.make_params(w["sigma2"], w["r"], w["t"], R, w["lmax_iters"], int(w["cap_frac"] * gm.n),
                       G.GRASS_FP32 if w["embed"] == "fp32" else G.GRASS_FP64, w["inner_tol"],
                       w["inner_maxit"])
    res["unit_mesh_1000"] = lsst_vs_mst(G, wm, Pm, gm, hm, vm, bm,
                                        "1000x1000 unit mesh, D = 1e-3 I; the step's densification "
                                        "parameters; PCG to 1e-3 (FP32 + FP64 refinement), tree "
                                        "only and with the sparsifier")
    return res


# ---------------------------------------------------------------- replicas

def replica_max(dist, v: float, device: str = "cuda") -> float:
    """Largest of v over the ranks of the process group (v itself alone)."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, units_per_step_per_rank: float, ms_per_step_max: float) -> float:
    """Whole-job throughput of `world` independent replicas timed together:
    the units all ranks processed per step over the slowest rank's step."""
    return world * units_per_step_per_rank / (ms_per_step_max / 1e3)


# ---------------------------------------------------------------- GPU arm

def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="grass", choices=["grass", "reference"])
    ap.add_argument("--workload", default="grid3d_100", choices=sorted(WORKLOADS))
    ap.add_argument("--family", default="pcg", choices=sorted(FAMILIES),
                    help="kernel family timed for the roofline object")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pcg-precond", default="multigrid", choices=["tree", "multigrid"],
                    help="the step's PCG preconditioner: the tree solve with one inner step on "
                         "the sparsifier, or one V-cycle of the sparsifier's multigrid")
    ap.add_argument("--no-breakdown", action="store_true")
    ap.add_argument("--profile-step", action="store_true",
                    help="run exactly one step and exit (for ncu launch lists)")
    ap.add_argument("--profile-amg", action="store_true",
                    help="one warm and one NVTX-ranged ('amgpcg') multigrid-preconditioned PCG solve "
                         "(FP32 + FP64 refinement, 1e-8) on the step's sparsifier, for ncu launch lists")
    ap.add_argument("--profile-kernel", choices=["cg", "cg16", "tree", "pcg", "amgpcg"], default=None,
                    help="one warm launch, then one timed launch of the kernel (for ncu captures)")
    ap.add_argument("--no-solve40m", action="store_true",
                    help="skip the 40M-unknown solve (solve_40m key of the line)")
    ap.add_argument("--serve", action="store_true",
                    help="run the serving benchmark instead and print its line")
    ap.add_argument("--solve40m-only", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=None,
                    help="arrivals per load level of --serve (default 1000)")
    ap.add_argument("--serve-grid-sms", type=int, default=0,
                    help="SMs of each request's cooperative kernels in --serve (0: all)")
    ap.add_argument("--serve-capacity-only", action="store_true",
                    help="--serve: measure the closed-burst capacity only")
    ap.add_argument("--batch", action="store_true",
                    help="run the 256-graph batch benchmark instead and print its line")
    ap.add_argument("--only-extra", default=None,
                    choices=["lsst_vs_mst", "c3_powerlaw", "densify_budget"],
                    help="run only the named measurement (outside any timed region) and print it")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the keys measured outside the timed region (per-round rates, "
                         "kappa check, FP64 path, PCG inner sweep, 64x64 latency, power-law "
                         "workload, hair comb)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import paper_1911_04382_gb300 as G

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    G.lib()   # fails loudly if the CUDA library is missing
    if args.serve or args.solve40m_only or args.batch:
        out = run_serve(G, args) if args.serve else (run_batch(G) if args.batch else solve_40m(G))
        out.update(n_gpus=world, data="synthetic")
        if rank == 0:
            print(json.dumps(out), flush=True)
        return 0
    g, h0, v0, b = make_inputs(w)
    stream = torch.cuda.current_stream()
    ctx = G.grass_ctx_create(stream)
    if args.pcg_precond == "multigrid":
        G.grass_ctx_set_param(ctx, "pcg_precond", 1)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, col, val = dev(g.rowptr), dev(g.col), dev(g.val)
    h0d, v0d, bd = dev(h0), dev(v0), dev(b)
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    embed_prec = G.GRASS_FP32 if w["embed"] == "fp32" else G.GRASS_FP64
    pcg_prec = G.GRASS_FP32 if w["pcg"] == "fp32" else G.GRASS_FP64
    cap = int(w["cap_frac"] * g.n)
    P = G.make_params(w["sigma2"], w["r"], w["t"], w["rounds"], w["lmax_iters"], cap, embed_prec,
                      w["inner_tol"], w["inner_maxit"])
    last = {}

    def step(rp, col, val, h0d, v0d, bd, x, before_densify=None):
        t0 = time.perf_counter()
        tree = G.grass_build_tree(ctx, rp, col, val, 0)
        t1 = time.perf_counter()
        if before_densify is not None:
            before_densify()
        S, st = G.grass_densify(ctx, tree, P, h0d, v0d)
        t2 = time.perf_counter()
        status, sst = G.grass_pcg_solve(ctx, S, bd, x, w["pcg_tol"], w["pcg_maxit"], pcg_prec,
                                        w["refine_tol"], w["pcg_inner_tol"], w["pcg_inner_maxit"])
        t3 = time.perf_counter()
        n_s, _ = G.grass_sparsifier_info(S)
        rounds = G.grass_tree_info(tree)[2]
        G.grass_sparsifier_destroy(S)
        G.grass_tree_destroy(tree)
        last.update(st=st.as_dict(), sst=sst.as_dict(), status=status, n_s=n_s, tree_rounds=rounds,
                    phase_ms={"tree": 1e3 * (t1 - t0), "densify": 1e3 * (t2 - t1),
                              "pcg": 1e3 * (t3 - t2)})
        return st.offtree_embedded

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v: float) -> float:
        return replica_max(dist, v, "cuda")

    if args.profile_kernel:
        return profile_kernel(G, ctx, args.profile_kernel, g, rp, col, val, v0d, w)

    if args.only_extra:
        fn = {"lsst_vs_mst": lambda: lsst_extras(G, w, P, g, h0d, v0d, bd),
              "c3_powerlaw": lambda: c3_powerlaw(G, peak_hbm()),
              "densify_budget": lambda: densify_budget(G, w, g, rp, col, val, bd)}[args.only_extra]
        print(json.dumps({args.only_extra: fn()}), flush=True)
        G.grass_ctx_destroy(ctx)
        return 0

    if args.profile_amg:
        tree = G.grass_build_tree(ctx, rp, col, val, 0)
        S, _ = G.grass_densify(ctx, tree, P, h0d, v0d)
        G.grass_ctx_set_param(ctx, "pcg_precond", 1)
        G.grass_pcg_solve(ctx, S, bd, x, w["pcg_tol"], w["pcg_maxit"], pcg_prec, w["refine_tol"],
                          w["pcg_inner_tol"], 0)                       # warm: builds the hierarchy
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("amgpcg")
        t0 = time.perf_counter()
        s_, ps = G.grass_pcg_solve(ctx, S, bd, x, w["pcg_tol"], w["pcg_maxit"], pcg_prec,
                                   w["refine_tol"], w["pcg_inner_tol"], 0)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_amg": True, "iters": ps.iters, "rel_resid_fp64": ps.rel_resid_fp64,
                          "ms": 1e3 * (time.perf_counter() - t0)}), flush=True)
        G.grass_sparsifier_destroy(S)
        G.grass_tree_destroy(tree)
        G.grass_ctx_destroy(ctx)
        return 0

    if args.profile_step:
        # the autotuner's choice first (as in the timed run), then one step
        # inside the NVTX range "step" (ncu --nvtx --nvtx-include "step/")
        t_tune = G.grass_build_tree(ctx, rp, col, val, 0)
        G.grass_autotune_rows(ctx, t_tune, w["r"], embed_prec)
        G.grass_tree_destroy(t_tune)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("step")
        e = step(rp, col, val, h0d, v0d, bd, x)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_step": True, "edges": e, "launches": G.grass_launch_count(ctx),
                          "phase_ms": last.get("phase_ms")}), flush=True)
        G.grass_ctx_destroy(ctx)
        return 0

    # row-kernel autotuner (SpMM launch variant and chunk width, heat form)
    # on this graph for the step's r and precision, before the warm-up
    t_tune = G.grass_build_tree(ctx, rp, col, val, 0)
    row_best, row_ms = G.grass_autotune_rows(ctx, t_tune, w["r"], embed_prec)
    G.grass_tree_destroy(t_tune)
    row_tune = {"spmm_chunk_cap": row_best[0], "spmm_variant": row_best[1],
                "heat_form": row_best[2], "spmm_ms": row_ms[0], "heat_ms": row_ms[1],
                "what": "grass_autotune_rows on the step's graph, r and precision, before the warm-up"}

    for _ in range(max(args.warmup, 0)):
        step(rp, col, val, h0d, v0d, bd, x)

    gpu_id = str(local)
    try:
        uuid = getattr(torch.cuda.get_device_properties(local), "uuid", None)
        if uuid is not None:
            gpu_id = "GPU-" + str(uuid) if not str(uuid).startswith("GPU-") else str(uuid)
    except Exception:
        pass
    clocks = ClockSampler(gpu_id)
    G.grass_kernel_timing_enable(ctx, FAMILIES[args.family])
    launches0 = G.grass_launch_count(ctx)
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    edges = 0
    for _ in range(args.steps):
        edges += step(rp, col, val, h0d, v0d, bd, x)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = G.grass_launch_count(ctx) - launches0
    kms, kl, kbytes = G.grass_kernel_timing_read(ctx)
    G.grass_kernel_timing_enable(ctx, 0)
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps)
    edges_per_step = edges / args.steps
    value = replica_value(world, edges_per_step, ms)

    # e2e: host (pinned) inputs copied in and the result copied out, every
    # step.  The copies run on a copy stream: the CSR first (the tree build
    # waits for it), then the start vectors and b, which the step waits for
    # only before densification, so they overlap the tree build
    host = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hp = [host(g.rowptr), host(g.col), host(g.val), host(h0), host(v0), host(b)]
    dbufs = [torch.empty_like(t, device="cuda") for t in hp]
    xh = torch.empty(g.n, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in hp)
    d2h = xh.numel() * xh.element_size()
    cstream = torch.cuda.Stream()
    ev_csr, ev_rest = torch.cuda.Event(), torch.cuda.Event()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e_edges = 0
    for _ in range(args.steps):
        cstream.wait_stream(stream)          # the previous step is done with the buffers
        with torch.cuda.stream(cstream):
            for d, h in zip(dbufs[:3], hp[:3]):
                d.copy_(h, non_blocking=True)
            ev_csr.record(cstream)
            for d, h in zip(dbufs[3:], hp[3:]):
                d.copy_(h, non_blocking=True)
            ev_rest.record(cstream)
        stream.wait_event(ev_csr)
        e_edges += step(*dbufs, x, before_densify=lambda: stream.wait_event(ev_rest))
        xh.copy_(x, non_blocking=True)
    e1.record(stream)
    barrier()
    e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    e2e = {"value": world * (e_edges / args.steps) / (e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e_ms}

    # per-family breakdown (one extra step per family, not part of value)
    breakdown = {}
    if not args.no_breakdown and rank == 0:
        for name, fam in FAMILIES.items():
            G.grass_kernel_timing_enable(ctx, fam)
            step(rp, col, val, h0d, v0d, bd, x)
            fms, fl, fb = G.grass_kernel_timing_read(ctx)
            breakdown[name] = {"ms_per_step": fms, "launches": fl,
                               "GBps": (fb / (fms / 1e3) / 1e9) if fms > 0 else None}
        G.grass_kernel_timing_enable(ctx, 0)

    peaks = measured_peaks()
    peak = peak_hbm()
    achieved = (kbytes / kl) / ((kms / kl) / 1e3) / 1e9 if kl and kms > 0 else None
    # DRAM traffic per launch from the committed ncu capture (dram bytes /
    # algorithmic bytes of the captured launch, times this run's algorithmic
    # bytes per launch); null when the kernel sources changed since
    traffic_note = None
    # the PCG family's kernel is the fused multigrid PCG under --pcg-precond multigrid
    fam_key = "amgpcg" if args.family == "pcg" and args.pcg_precond == "multigrid" else args.family
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        rec = tr.get(args.workload, {}).get(fam_key)
        if rec and rec.get("sources") == kernel_sources_hash() and kl:
            traffic_note = rec["dram_bytes"] / rec["algorithmic_bytes"] * (kbytes / kl)
    except Exception:
        pass
    roofline = {
        "kernel": fam_key, "bound": "hbm", "achieved": achieved, "peak": peak,
        "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
        "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback 6800 GB/s",
        "traffic": traffic_note, "launches_timed": kl,
        "algorithmic_bytes_per_launch": (kbytes / kl) if kl else None,
        "avg_launch_us": (1e3 * kms / kl) if kl else None,
    }

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        reps, tot, e = 0, 0.0, 0
        while tot < 8.0 and reps < 8:
            e, s = oracle_sample(w, g, h0, v0)
            tot += s
            reps += 1
        cpu = {"value": e / (tot / reps), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{reps} x (oracle extraction + Kruskal tree + round-1 lambda estimates "
                         f"+ FP64 embedding/heat/filter of all {e} off-tree edges), single thread"}

    extras = {}
    if rank == 0 and not args.no_extras and args.workload == "grid3d_100":
        for name, fn in (("c2", lambda: c2_extras(G, ctx, w, g, rp, col, val, h0d, v0d, bd, P, peak,
                                                      args.pcg_precond == "multigrid")),
                         ("c1_latency", lambda: c1_latency(G)),
                         ("c3_powerlaw", lambda: c3_powerlaw(G, peak)),
                         ("hair_comb", lambda: hair_comb(G)),
                         ("lsst_vs_mst", lambda: lsst_extras(G, w, P, g, h0d, v0d, bd)),
                         ("densify_budget", lambda: densify_budget(G, w, g, rp, col, val, bd)),
                         ("partition_mesh_1m", lambda: partition_mesh(G))):
            try:
                r_ = fn()
                if name == "c2":
                    extras.update(r_)
                else:
                    extras[name] = r_
            except Exception as ex:          # reported, never fatal for the line
                extras[name] = {"error": f"{type(ex).__name__}: {ex}"[:300]}
        if last.get("st"):
            extras["per_round"] = per_round(last["st"], g, w, peak)

    s40 = None
    if rank == 0 and not args.no_solve40m and args.workload == "grid3d_100":
        try:
            s40 = solve_40m(G)
        except Exception as ex:          # reported, never fatal for the line
            s40 = {"error": f"{type(ex).__name__}: {ex}"[:300]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if w["embed"] == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": describe(w, g), "name": args.workload, "n": g.n, "m": g.m,
                       "nnz": g.nnz, "per_round_cap": cap,
                       "l2": "inputs larger than L2 (CSR + start vectors resident: "
                             f"{(g.nnz * 12 + h0.nbytes + v0.nbytes) / 1e6:.0f} MB)",
                       "pcg_preconditioner": args.pcg_precond,
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clk, "edges_embedded_per_step": edges_per_step,
            "phase_ms": last.get("phase_ms"), "densify": last.get("st"), "pcg": last.get("sst"),
            "sparsifier_edges": last.get("n_s"), "tree_factor_rounds": last.get("tree_rounds"),
            "kernels": breakdown, "solve_40m": s40, "row_autotune": row_tune,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    G.grass_ctx_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
