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

FAMILIES = {"spmm_g": 1, "spmm_s": 2, "heat": 3, "tree": 4, "cg": 5}


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
                  "paper_1911_04382_gb300/csrc/common.cuh"]


def kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for s in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, s), "rb").read())
    return h.hexdigest()[:16]


def profile_kernel(G, ctx, which, g, rp, col, val, v0d, w) -> int:
    """One warm and one timed launch of the fused inner CG (exactly 30
    iterations, r = 1, FP32, sparsifier = tree + every 197th off-tree edge)
    or of the tree solve (r = 16, FP32); prints its algorithmic bytes."""
    import torch
    tree = G.grass_build_tree(ctx, rp, col, val, 0)
    if which == "cg":
        S = G.grass_sparsifier_create(ctx, tree)
        _, moff = G.grass_sparsifier_info(S)
        ids = torch.empty(moff, dtype=torch.int64, device="cuda")
        G.grass_sparsifier_offtree(ctx, S, ids)
        G.grass_sparsifier_add(ctx, S, ids[::197].contiguous())
        run = lambda: G.grass_lambda_max(ctx, S, v0d[:g.n], 1, G.GRASS_FP32, 0.0, 30)
        fam, units = G.GRASS_KF_CG, "30 iterations, r=1"
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


# ---------------------------------------------------------------- GPU arm

def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="grass", choices=["grass", "reference"])
    ap.add_argument("--workload", default="grid3d_100", choices=sorted(WORKLOADS))
    ap.add_argument("--family", default="cg", choices=sorted(FAMILIES),
                    help="kernel family timed for the roofline object")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-breakdown", action="store_true")
    ap.add_argument("--profile-step", action="store_true",
                    help="run exactly one step and exit (for ncu launch lists)")
    ap.add_argument("--profile-kernel", choices=["cg", "tree"], default=None,
                    help="one warm launch, then one timed launch of the kernel (for ncu captures)")
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
    g, h0, v0, b = make_inputs(w)
    stream = torch.cuda.current_stream()
    ctx = G.grass_ctx_create(stream)
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

    def step(rp, col, val, h0d, v0d, bd, x):
        t0 = time.perf_counter()
        tree = G.grass_build_tree(ctx, rp, col, val, 0)
        t1 = time.perf_counter()
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
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    if args.profile_kernel:
        return profile_kernel(G, ctx, args.profile_kernel, g, rp, col, val, v0d, w)

    if args.profile_step:
        e = step(rp, col, val, h0d, v0d, bd, x)
        torch.cuda.synchronize()
        print(json.dumps({"profile_step": True, "edges": e, "launches": G.grass_launch_count(ctx),
                          "phase_ms": last.get("phase_ms")}), flush=True)
        G.grass_ctx_destroy(ctx)
        return 0

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
    value = world * edges_per_step / (ms / 1e3)

    # e2e: host (pinned) inputs copied in and the result copied out, every step
    host = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hp = [host(g.rowptr), host(g.col), host(g.val), host(h0), host(v0), host(b)]
    dbufs = [torch.empty_like(t, device="cuda") for t in hp]
    xh = torch.empty(g.n, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in hp)
    d2h = xh.numel() * xh.element_size()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e_edges = 0
    for _ in range(args.steps):
        for d, h in zip(dbufs, hp):
            d.copy_(h, non_blocking=True)
        e_edges += step(*dbufs, x)
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

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = (kbytes / kl) / ((kms / kl) / 1e3) / 1e9 if kl and kms > 0 else None
    # DRAM traffic per launch from the committed ncu capture (dram bytes /
    # algorithmic bytes of the captured launch, times this run's algorithmic
    # bytes per launch); null when the kernel sources changed since
    traffic_note = None
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        rec = tr.get(args.workload, {}).get(args.family)
        if rec and rec.get("sources") == kernel_sources_hash() and kl:
            traffic_note = rec["dram_bytes"] / rec["algorithmic_bytes"] * (kbytes / kl)
    except Exception:
        pass
    roofline = {
        "kernel": args.family, "bound": "hbm", "achieved": achieved, "peak": peak,
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
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clk, "edges_embedded_per_step": edges_per_step,
            "phase_ms": last.get("phase_ms"), "densify": last.get("st"), "pcg": last.get("sst"),
            "sparsifier_edges": last.get("n_s"), "tree_factor_rounds": last.get("tree_rounds"),
            "kernels": breakdown,
        }
        print(json.dumps(line), flush=True)
    G.grass_ctx_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
