"""ctypes binding of libgrass.so (include/grass.h), same names as the C ABI.

Argument marshalling only: device buffers are torch tensors (or raw integer
addresses), host results come back as Python values.  Every GPU step runs in
the library's CUDA kernels; there is no fallback path.  A missing library is
an error: build it with ``paper_1911_04382_gb300.build()``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from .build import LIB

GRASS_OK = 0
GRASS_ERR_INVALID = 1
GRASS_ERR_NOT_SDD = 2
GRASS_ERR_DISCONNECTED = 3
GRASS_ERR_OOM = 4
GRASS_ERR_NOT_CONVERGED = 5
GRASS_ERR_TIMEOUT = 6
GRASS_ERR_CUDA = 7
GRASS_FP64 = 0
GRASS_FP32 = 1
GRASS_MAX_ROUNDS = 16

_STATUS = {0: "OK", 1: "INVALID", 2: "NOT_SDD", 3: "DISCONNECTED", 4: "OOM",
           5: "NOT_CONVERGED", 6: "TIMEOUT", 7: "CUDA"}


class GrassError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: GRASS_ERR_{_STATUS.get(status, status)}: {msg}")
        self.status = status


class grass_csr_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class grass_params_t(C.Structure):
    _fields_ = [("sigma2", C.c_double), ("r", C.c_int), ("t", C.c_int), ("max_rounds", C.c_int),
                ("lmax_iters", C.c_int), ("max_add_per_round", C.c_int64),
                ("embed_prec", C.c_int), ("inner_tol", C.c_double), ("inner_maxit", C.c_int)]


_R = GRASS_MAX_ROUNDS


class grass_sparsify_stats_t(C.Structure):
    _fields_ = [("rounds", C.c_int), ("stopped_similar", C.c_int), ("added", C.c_int64),
                ("offtree_embedded", C.c_int64), ("added_round", C.c_int64 * _R),
                ("embedded_round", C.c_int64 * _R), ("lmin_est", C.c_double * _R),
                ("lmax_est", C.c_double * _R), ("theta", C.c_double * _R),
                ("heat_max", C.c_double * _R), ("inner_iters", C.c_int64),
                ("ms_estimate", C.c_double), ("ms_embed", C.c_double), ("ms_filter", C.c_double),
                ("ms_update", C.c_double), ("ms_total", C.c_double),
                ("ms_embed_round", C.c_double * _R), ("lmax_capped", C.c_int64 * _R)]

    def as_dict(self) -> dict:
        k = max(self.rounds, 1 if self.stopped_similar else 0)
        k = min(max(k, self.rounds + (1 if self.stopped_similar else 0)), _R)
        return {
            "rounds": self.rounds, "stopped_similar": bool(self.stopped_similar),
            "added": self.added, "offtree_embedded": self.offtree_embedded,
            "added_round": list(self.added_round[:self.rounds]),
            "embedded_round": list(self.embedded_round[:self.rounds]),
            "lmin_est": list(self.lmin_est[:k]), "lmax_est": list(self.lmax_est[:k]),
            "theta": list(self.theta[:self.rounds]), "heat_max": list(self.heat_max[:self.rounds]),
            "inner_iters": self.inner_iters, "ms_estimate": self.ms_estimate,
            "ms_embed": self.ms_embed, "ms_filter": self.ms_filter, "ms_update": self.ms_update,
            "ms_total": self.ms_total, "ms_embed_round": list(self.ms_embed_round[:self.rounds]),
            "lmax_capped": list(self.lmax_capped[:k]),
        }


class grass_solve_stats_t(C.Structure):
    _fields_ = [("iters", C.c_int), ("refinements", C.c_int), ("inner_iters", C.c_int64),
                ("rel_resid_fp64", C.c_double), ("ms", C.c_double)]

    def as_dict(self) -> dict:
        return {"iters": self.iters, "refinements": self.refinements,
                "inner_iters": self.inner_iters, "rel_resid_fp64": self.rel_resid_fp64,
                "ms": self.ms}


class grass_fiedler_stats_t(C.Structure):
    _fields_ = [("iters_done", C.c_int), ("pcg_iters", C.c_int64), ("worst_rel_resid", C.c_double),
                ("n_pos", C.c_int64), ("n_neg", C.c_int64), ("rayleigh", C.c_double),
                ("ms", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class grass_lsst_stats_t(C.Structure):
    _fields_ = [("classes", C.c_int32), ("levels", C.c_int64), ("rounds", C.c_int64),
                ("ms", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class grass_request_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("h0", C.c_void_p), ("v0", C.c_void_p), ("b", C.c_void_p),
                ("x", C.c_void_p), ("params", grass_params_t), ("tol", C.c_double),
                ("maxit", C.c_int), ("pcg_prec", C.c_int), ("refine_tol", C.c_double),
                ("pcg_inner_tol", C.c_double), ("pcg_inner_maxit", C.c_int)]


class grass_result_t(C.Structure):
    _fields_ = [("status", C.c_int), ("error", C.c_char * 128),
                ("sparsify", grass_sparsify_stats_t), ("solve", grass_solve_stats_t),
                ("footprint_bytes", C.c_int64), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("ms_h2d", C.c_double), ("ms_tree", C.c_double),
                ("ms_densify", C.c_double), ("ms_pcg", C.c_double), ("slot", C.c_int),
                ("in_flight_at_admit", C.c_int)]


_lib = None
_lock = threading.Lock()
_vp, _i64, _i32, _d = C.c_void_p, C.c_int64, C.c_int32, C.c_double


def lib():
    """Load libgrass.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(f"CUDA library {LIB} is missing: run paper_1911_04382_gb300.build()")
            L = C.CDLL(LIB)
            sig = {
                "grass_ctx_create": [C.POINTER(_vp), _vp],
                "grass_ctx_set_stream": [_vp, _vp],
                "grass_kernel_timing_enable": [_vp, C.c_int],
                "grass_ctx_set_wait_limit": [_vp, _i64, C.c_int],
                "grass_ctx_set_param": [_vp, C.c_char_p, _i64],
                "grass_tree_schedule_info": [_vp, C.POINTER(_i64), C.POINTER(_i64),
                                             C.POINTER(_i64), _i64],
                "grass_kernel_timing_read": [_vp, C.POINTER(_d), C.POINTER(_i64), C.POINTER(_d)],
                "grass_build_tree": [_vp, C.POINTER(grass_csr_t), _i32, C.POINTER(_vp)],
                "grass_tree_from_edges": [_vp, C.POINTER(grass_csr_t), _vp, _i32, C.POINTER(_vp)],
                "grass_build_lsst": [_vp, C.POINTER(grass_csr_t), C.c_uint64, _i32, C.POINTER(_vp),
                                     C.POINTER(grass_lsst_stats_t)],
                "grass_tree_stretch": [_vp, _vp, _vp, C.POINTER(_d)],
                "grass_autotune_rows": [_vp, _vp, C.c_int, C.c_int, C.POINTER(_i32), C.POINTER(_d)],
                "grass_sparsifier_edges": [_vp, C.POINTER(_i64), _i64, C.POINTER(_i64)],
                "grass_tree_info": [_vp, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64)],
                "grass_tree_graph": [_vp, _vp, _vp, _vp, _vp, _vp],
                "grass_tree_edges": [_vp, _vp, _vp],
                "grass_tree_solve": [_vp, _vp, C.c_int, C.c_int, C.c_int, _vp, _vp],
                "grass_tree_solve_noalloc": [_vp, _vp, C.c_int, C.c_int, C.c_int, _vp, _vp],
                "grass_spmm": [_vp, _vp, C.c_int, C.c_int, _vp, _vp],
                "grass_sparsifier_create": [_vp, _vp, C.POINTER(_vp)],
                "grass_sparsifier_add": [_vp, _vp, _vp, _i64],
                "grass_sparsifier_info": [_vp, C.POINTER(_i64), C.POINTER(_i64)],
                "grass_sparsifier_mask": [_vp, _vp, _vp],
                "grass_sparsifier_offtree": [_vp, _vp, _vp],
                "grass_embed": [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _d, C.c_int, _vp, _vp,
                                C.POINTER(_d)],
                "grass_lambda_min": [_vp, _vp, C.POINTER(_d)],
                "grass_lambda_max": [_vp, _vp, _vp, C.c_int, C.c_int, _d, C.c_int, C.POINTER(_d)],
                "grass_filter": [_vp, _vp, _vp, C.c_int, _d, _d, _d, C.c_int, _i64, _vp,
                                 C.POINTER(_i64), C.POINTER(_d)],
                "grass_filter_similar": [_vp, _vp, _vp, C.c_int, _d, _d, _d, C.c_int, _i64, _vp,
                                         C.POINTER(_i64), C.POINTER(_d)],
                "grass_densify": [_vp, _vp, C.POINTER(grass_params_t), _vp, _vp, C.POINTER(_vp),
                                  C.POINTER(grass_sparsify_stats_t)],
                "grass_pcg_solve": [_vp, _vp, _vp, _vp, _d, C.c_int, C.c_int, _d, _d, C.c_int,
                                    C.POINTER(grass_solve_stats_t)],
                "grass_fiedler": [_vp, _vp, _vp, C.c_int, _d, C.c_int, C.c_int, C.c_int, _vp, _vp,
                                  C.POINTER(grass_fiedler_stats_t)],
                "grass_build_forest": [_vp, C.POINTER(grass_csr_t), _i64, C.POINTER(_i64),
                                       C.POINTER(_vp)],
                "grass_tree_segments": [_vp, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64)],
                "grass_densify_batch": [_vp, _vp, C.POINTER(grass_params_t), _vp, _vp,
                                        C.POINTER(_vp), C.POINTER(grass_sparsify_stats_t),
                                        C.POINTER(_d)],
                "grass_pcg_solve_batch": [_vp, _vp, _vp, _vp, _d, C.c_int, C.c_int, C.c_int,
                                          C.POINTER(grass_solve_stats_t), C.POINTER(_i32),
                                          C.POINTER(_d)],
                "grass_autotune": [_vp, _vp, C.c_int, C.c_int, C.POINTER(_i64), C.POINTER(_d)],
                "grass_server_create": [C.c_int, C.c_int, _i64, C.POINTER(_vp)],
                "grass_server_set_param": [_vp, C.c_char_p, _i64],
                "grass_server_submit": [_vp, C.POINTER(grass_request_t), C.POINTER(_i64)],
                "grass_server_wait": [_vp, _i64, C.POINTER(grass_result_t)],
                "grass_server_stats": [_vp, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64),
                                       C.POINTER(_i64)],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int
            L.grass_server_footprint.argtypes = [_i64, _i64, C.c_int, C.c_int]
            L.grass_server_footprint.restype = C.c_int64
            L.grass_server_budget.argtypes = [_vp]
            L.grass_server_budget.restype = C.c_int64
            for name in ("grass_ctx_destroy", "grass_tree_destroy", "grass_sparsifier_destroy",
                         "grass_server_destroy"):
                getattr(L, name).argtypes = [_vp]
                getattr(L, name).restype = None
            L.grass_last_error.argtypes = [_vp]
            L.grass_last_error.restype = C.c_char_p
            L.grass_launch_count.argtypes = [_vp]
            L.grass_launch_count.restype = C.c_int64
            _lib = L
    return _lib


def _p(x):
    """Device address of a tensor, an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(ctx, st: int, where: str, allow=()):
    if st != GRASS_OK and st not in allow:
        msg = lib().grass_last_error(ctx).decode() if ctx else ""
        raise GrassError(st, where, msg)
    return st


# ---------------------------------------------------------------- context

def grass_ctx_create(stream=None) -> int:
    out = _vp()
    st = lib().grass_ctx_create(C.byref(out), _stream(stream))
    if st != GRASS_OK:
        raise GrassError(st, "grass_ctx_create", "context creation failed")
    return out.value


def grass_ctx_destroy(ctx: int) -> None:
    lib().grass_ctx_destroy(ctx)


def grass_ctx_set_stream(ctx: int, stream=None) -> None:
    _check(ctx, lib().grass_ctx_set_stream(ctx, _stream(stream)), "grass_ctx_set_stream")


def grass_last_error(ctx: int) -> str:
    return lib().grass_last_error(ctx).decode()


def grass_launch_count(ctx: int) -> int:
    return int(lib().grass_launch_count(ctx))


def grass_ctx_set_param(ctx: int, name: str, value: int) -> None:
    _check(ctx, lib().grass_ctx_set_param(ctx, name.encode(), int(value)), "grass_ctx_set_param")


def grass_tree_schedule_info(tree: int, cap: int = 4096):
    """Per-round (eliminated, receivers, contributions) lists."""
    n, m, rounds = grass_tree_info(tree)
    k = min(rounds, cap)
    a, b, c = (_i64 * max(k, 1))(), (_i64 * max(k, 1))(), (_i64 * max(k, 1))()
    _check(None, lib().grass_tree_schedule_info(tree, a, b, c, k), "grass_tree_schedule_info")
    return list(a[:k]), list(b[:k]), list(c[:k])


def grass_ctx_set_wait_limit(ctx: int, polls: int = 0, hold_barriers: int = 0) -> None:
    _check(ctx, lib().grass_ctx_set_wait_limit(ctx, int(polls), int(hold_barriers)),
           "grass_ctx_set_wait_limit")


GRASS_KF_NONE, GRASS_KF_SPMM_G, GRASS_KF_SPMM_S, GRASS_KF_HEAT, GRASS_KF_TREE, GRASS_KF_CG = 0, 1, 2, 3, 4, 5
GRASS_KF_PCG, GRASS_KF_SPMM_BLK = 6, 7


def grass_kernel_timing_enable(ctx: int, family: int) -> None:
    _check(ctx, lib().grass_kernel_timing_enable(ctx, int(family)), "grass_kernel_timing_enable")


def grass_kernel_timing_read(ctx: int) -> tuple[float, int, float]:
    """(summed event ms, timed launches, summed algorithmic bytes)."""
    ms, nl, by = _d(0.0), _i64(0), _d(0.0)
    _check(ctx, lib().grass_kernel_timing_read(ctx, C.byref(ms), C.byref(nl), C.byref(by)),
           "grass_kernel_timing_read")
    return ms.value, nl.value, by.value


# ---------------------------------------------------------------- tree

def grass_build_tree(ctx: int, rowptr, col, val, ground: int = 0, n: int | None = None,
                     nnz: int | None = None) -> int:
    """rowptr (int64 [n+1]), col (int32 [nnz]), val (float64 [nnz]) on the device."""
    A = grass_csr_t()
    A.n = int(rowptr.numel() - 1) if n is None else n
    A.nnz = int(col.numel()) if nnz is None else nnz
    A.rowptr, A.col, A.val = _p(rowptr), _p(col), _p(val)
    out = _vp()
    _check(ctx, lib().grass_build_tree(ctx, C.byref(A), int(ground), C.byref(out)),
           "grass_build_tree")
    return out.value


def grass_tree_from_edges(ctx: int, rowptr, col, val, tree_eids, ground: int = 0) -> int:
    """grass_build_tree with the caller's spanning tree: tree_eids (device
    int64, n-1 edge ids)."""
    A = grass_csr_t()
    A.n = int(rowptr.numel() - 1)
    A.nnz = int(col.numel())
    A.rowptr, A.col, A.val = _p(rowptr), _p(col), _p(val)
    out = _vp()
    _check(ctx, lib().grass_tree_from_edges(ctx, C.byref(A), _p(tree_eids), int(ground),
                                            C.byref(out)), "grass_tree_from_edges")
    return out.value


def grass_build_lsst(ctx: int, rowptr, col, val, seed: int = 1, ground: int = 0) -> tuple[int, dict]:
    """grass_build_tree with the low-stretch tree of the given seed; returns
    (tree handle, stats dict)."""
    A = grass_csr_t()
    A.n = int(rowptr.numel() - 1)
    A.nnz = int(col.numel())
    A.rowptr, A.col, A.val = _p(rowptr), _p(col), _p(val)
    out = _vp()
    st = grass_lsst_stats_t()
    _check(ctx, lib().grass_build_lsst(ctx, C.byref(A), C.c_uint64(int(seed) & (2**64 - 1)),
                                       int(ground), C.byref(out), C.byref(st)), "grass_build_lsst")
    return out.value, st.as_dict()


def grass_tree_stretch(ctx: int, tree: int, stretch=None) -> float:
    """Per-edge stretch into stretch (device float64 [m], optional); returns
    the total stretch st_T(G)."""
    tot = _d(0.0)
    _check(ctx, lib().grass_tree_stretch(ctx, tree, _p(stretch), C.byref(tot)),
           "grass_tree_stretch")
    return tot.value


def grass_autotune_rows(ctx: int, tree: int, r: int, prec: int) -> tuple[list, list]:
    """Row-kernel autotuner: returns ([chunk cap, SpMM variant, heat form],
    [SpMM ms, heat ms])."""
    best = (_i32 * 3)()
    ms = (_d * 2)()
    _check(ctx, lib().grass_autotune_rows(ctx, tree, int(r), int(prec), best, ms),
           "grass_autotune_rows")
    return list(best), list(ms)


def grass_tree_destroy(tree: int) -> None:
    lib().grass_tree_destroy(tree)


def grass_tree_info(tree: int) -> tuple[int, int, int]:
    n, m, r = _i64(), _i64(), _i64()
    _check(None, lib().grass_tree_info(tree, C.byref(n), C.byref(m), C.byref(r)), "grass_tree_info")
    return n.value, m.value, r.value


def grass_tree_graph(ctx, tree, eu=None, ev=None, ew=None, D=None) -> None:
    _check(ctx, lib().grass_tree_graph(ctx, tree, _p(eu), _p(ev), _p(ew), _p(D)), "grass_tree_graph")


def grass_tree_edges(ctx, tree, in_tree) -> None:
    _check(ctx, lib().grass_tree_edges(ctx, tree, _p(in_tree)), "grass_tree_edges")


def grass_tree_solve(ctx, tree, with_D: int, r: int, prec: int, B, X) -> None:
    _check(ctx, lib().grass_tree_solve(ctx, tree, int(with_D), r, prec, _p(B), _p(X)),
           "grass_tree_solve")


def grass_tree_solve_noalloc(ctx, tree, with_D: int, r: int, prec: int, B, X) -> None:
    """grass_tree_solve without any device allocation (scratch compiled into
    the library); for callers that must not allocate device memory."""
    _check(ctx, lib().grass_tree_solve_noalloc(ctx, tree, int(with_D), r, prec, _p(B), _p(X)),
           "grass_tree_solve_noalloc")


def grass_spmm(ctx, tree, r: int, prec: int, X, Y) -> None:
    _check(ctx, lib().grass_spmm(ctx, tree, r, prec, _p(X), _p(Y)), "grass_spmm")


# ---------------------------------------------------------------- sparsifier

def grass_sparsifier_create(ctx, tree) -> int:
    out = _vp()
    _check(ctx, lib().grass_sparsifier_create(ctx, tree, C.byref(out)), "grass_sparsifier_create")
    return out.value


def grass_sparsifier_destroy(S) -> None:
    lib().grass_sparsifier_destroy(S)


def grass_sparsifier_add(ctx, S, eids, count: int | None = None) -> None:
    cnt = int(eids.numel()) if count is None else int(count)
    _check(ctx, lib().grass_sparsifier_add(ctx, S, _p(eids), cnt), "grass_sparsifier_add")


def grass_sparsifier_info(S) -> tuple[int, int]:
    a, b = _i64(), _i64()
    _check(None, lib().grass_sparsifier_info(S, C.byref(a), C.byref(b)), "grass_sparsifier_info")
    return a.value, b.value


def grass_sparsifier_mask(ctx, S, in_s) -> None:
    _check(ctx, lib().grass_sparsifier_mask(ctx, S, _p(in_s)), "grass_sparsifier_mask")


def grass_sparsifier_edges(S, cap: int | None = None):
    """Host export: (ids of the edges in S in increasing order as a numpy
    int64 array of min(cap, count) entries, count).  cap None: all."""
    import numpy as np
    if cap is None:
        ne, _ = grass_sparsifier_info(S)
        cap = ne
    out = np.empty(max(int(cap), 1), dtype=np.int64)
    cnt = _i64(0)
    _check(None, lib().grass_sparsifier_edges(S, out.ctypes.data_as(C.POINTER(_i64)), int(cap),
                                              C.byref(cnt)), "grass_sparsifier_edges")
    return out[:min(int(cap), cnt.value)].copy(), cnt.value


def grass_sparsifier_offtree(ctx, S, eids) -> None:
    _check(ctx, lib().grass_sparsifier_offtree(ctx, S, _p(eids)), "grass_sparsifier_offtree")


# ---------------------------------------------------------------- embed / filter

def grass_embed(ctx, S, h0, r: int, t: int, prec: int, inner_tol: float = 1e-10,
                inner_maxit: int = 1000, H_out=None, heat=None) -> float:
    hm = _d(0.0)
    _check(ctx, lib().grass_embed(ctx, S, _p(h0), r, t, prec, inner_tol, inner_maxit, _p(H_out),
                                  _p(heat), C.byref(hm)), "grass_embed")
    return hm.value


def grass_lambda_min(ctx, S) -> float:
    v = _d(0.0)
    _check(ctx, lib().grass_lambda_min(ctx, S, C.byref(v)), "grass_lambda_min")
    return v.value


def grass_lambda_max(ctx, S, v0, iters: int, prec: int, inner_tol: float = 1e-10,
                     inner_maxit: int = 1000) -> float:
    v = _d(0.0)
    _check(ctx, lib().grass_lambda_max(ctx, S, _p(v0), iters, prec, inner_tol, inner_maxit,
                                       C.byref(v)), "grass_lambda_max")
    return v.value


def grass_filter(ctx, S, heat, prec: int, sigma2: float, lmin: float, lmax: float, t: int,
                 cap: int, accepted) -> tuple[int, float]:
    na, th = _i64(0), _d(0.0)
    _check(ctx, lib().grass_filter(ctx, S, _p(heat), prec, sigma2, lmin, lmax, t, int(cap),
                                   _p(accepted), C.byref(na), C.byref(th)), "grass_filter")
    return na.value, th.value


def grass_filter_similar(ctx, S, heat, prec: int, sigma2: float, lmin: float, lmax: float,
                         t: int, cap: int, accepted) -> tuple[int, float]:
    na, th = _i64(0), _d(0.0)
    _check(ctx, lib().grass_filter_similar(ctx, S, _p(heat), prec, sigma2, lmin, lmax, t, int(cap),
                                           _p(accepted), C.byref(na), C.byref(th)),
           "grass_filter_similar")
    return na.value, th.value


def grass_fiedler(ctx, S, x0, iters: int, tol: float, maxit: int, prec: int = GRASS_FP64,
                  inner_maxit: int = 1, u_out=None, side_out=None):
    """(status, grass_fiedler_stats_t); NOT_CONVERGED is returned, not raised."""
    st = grass_fiedler_stats_t()
    s = _check(ctx, lib().grass_fiedler(ctx, S, _p(x0), int(iters), float(tol), int(maxit), prec,
                                        int(inner_maxit), _p(u_out), _p(side_out), C.byref(st)),
               "grass_fiedler", allow=(GRASS_ERR_NOT_CONVERGED,))
    return s, st


# ---------------------------------------------------------------- densify / solve

def make_params(sigma2: float, r: int, t: int, max_rounds: int, lmax_iters: int = 8,
                max_add_per_round: int = 0, embed_prec: int = GRASS_FP64,
                inner_tol: float = 1e-10, inner_maxit: int = 1000) -> grass_params_t:
    P = grass_params_t()
    P.sigma2, P.r, P.t, P.max_rounds, P.lmax_iters = sigma2, r, t, max_rounds, lmax_iters
    P.max_add_per_round, P.embed_prec = max_add_per_round, embed_prec
    P.inner_tol, P.inner_maxit = inner_tol, inner_maxit
    return P


def grass_densify(ctx, tree, params: grass_params_t, h0, v0):
    """Returns (sparsifier handle, grass_sparsify_stats_t)."""
    out = _vp()
    st = grass_sparsify_stats_t()
    _check(ctx, lib().grass_densify(ctx, tree, C.byref(params), _p(h0), _p(v0), C.byref(out),
                                    C.byref(st)), "grass_densify")
    return out.value, st


def grass_pcg_solve(ctx, S, b, x, tol: float, maxit: int, prec: int, refine_tol: float = 1e-3,
                    inner_tol: float = 1e-6, inner_maxit: int = 50):
    """Returns (status, grass_solve_stats_t); NOT_CONVERGED is returned, not raised."""
    st = grass_solve_stats_t()
    s = _check(ctx, lib().grass_pcg_solve(ctx, S, _p(b), _p(x), tol, maxit, prec, refine_tol,
                                          inner_tol, inner_maxit, C.byref(st)),
               "grass_pcg_solve", allow=(GRASS_ERR_NOT_CONVERGED,))
    return s, st


# ---------------------------------------------------------------- serving

def grass_server_footprint(n: int, nnz: int, r: int, rounds: int) -> int:
    return int(lib().grass_server_footprint(n, nnz, r, rounds))


def grass_server_create(device: int = 0, slots: int = 4, hbm_budget: int = 0) -> int:
    out = _vp()
    _check(None, lib().grass_server_create(device, slots, int(hbm_budget), C.byref(out)),
           "grass_server_create")
    return out.value


def grass_server_budget(srv) -> int:
    return int(lib().grass_server_budget(srv))


def grass_server_destroy(srv) -> None:
    lib().grass_server_destroy(srv)


def grass_server_stats(srv) -> dict:
    v = [_i64(0) for _ in range(4)]
    _check(None, lib().grass_server_stats(srv, *[C.byref(a) for a in v]), "grass_server_stats")
    return dict(zip(("in_use", "queued", "running", "max_running"), (a.value for a in v)))


def grass_server_set_param(srv, name: str, value: int) -> None:
    _check(None, lib().grass_server_set_param(srv, name.encode(), int(value)),
           "grass_server_set_param")


class Server:
    """grass_server_* with the host arrays of each request kept alive until
    its result has been collected (the library reads them on admission)."""

    def __init__(self, device: int = 0, slots: int = 4, hbm_budget: int = 0):
        self.handle = grass_server_create(device, slots, hbm_budget)
        self._keep = {}
        self._mu = threading.Lock()

    def submit(self, rowptr, col, val, h0, v0, b, x, params: grass_params_t, tol: float,
               maxit: int, pcg_prec: int, refine_tol: float, pcg_inner_tol: float,
               pcg_inner_maxit: int) -> int:
        """numpy host arrays: rowptr int64, col int32, val/h0/v0/b/x float64 (x is written)."""
        arrs = (rowptr, col, val, h0, v0, b, x)
        q = grass_request_t()
        q.n, q.nnz = rowptr.shape[0] - 1, col.shape[0]
        q.rowptr, q.col, q.val, q.h0, q.v0, q.b, q.x = (a.ctypes.data for a in arrs)
        q.params = params
        q.tol, q.maxit, q.pcg_prec = tol, maxit, pcg_prec
        q.refine_tol, q.pcg_inner_tol, q.pcg_inner_maxit = refine_tol, pcg_inner_tol, pcg_inner_maxit
        t = _i64(0)
        _check(None, lib().grass_server_submit(self.handle, C.byref(q), C.byref(t)),
               "grass_server_submit")
        with self._mu:
            self._keep[t.value] = arrs
        return t.value

    def wait(self, ticket: int) -> grass_result_t:
        res = grass_result_t()
        _check(None, lib().grass_server_wait(self.handle, ticket, C.byref(res)), "grass_server_wait")
        with self._mu:
            self._keep.pop(ticket, None)
        return res

    def stats(self) -> dict:
        return grass_server_stats(self.handle)

    def set_param(self, name: str, value: int) -> None:
        grass_server_set_param(self.handle, name, value)

    def budget(self) -> int:
        return grass_server_budget(self.handle)

    def close(self) -> None:
        if self.handle:
            grass_server_destroy(self.handle)
            self.handle = None


def grass_server_submit(srv, req: grass_request_t) -> int:
    """Raw submit of a filled grass_request_t (the caller keeps its host
    arrays alive until grass_server_wait returns); Server.submit does that."""
    t = _i64(0)
    _check(None, lib().grass_server_submit(srv, C.byref(req), C.byref(t)), "grass_server_submit")
    return t.value


def grass_server_wait(srv, ticket: int) -> grass_result_t:
    res = grass_result_t()
    _check(None, lib().grass_server_wait(srv, ticket, C.byref(res)), "grass_server_wait")
    return res


# ---------------------------------------------------------------- batching

def grass_build_forest(ctx, rowptr, col, val, seg_off) -> int:
    """Union CSR on the device (as grass_build_tree); seg_off: host sequence
    of nseg+1 row offsets."""
    A = grass_csr_t()
    A.n, A.nnz = int(rowptr.numel() - 1), int(col.numel())
    A.rowptr, A.col, A.val = _p(rowptr), _p(col), _p(val)
    off = (_i64 * len(seg_off))(*[int(v) for v in seg_off])
    out = _vp()
    _check(ctx, lib().grass_build_forest(ctx, C.byref(A), len(seg_off) - 1, off, C.byref(out)),
           "grass_build_forest")
    return out.value


def grass_tree_segments(tree) -> tuple[list[int], list[int]]:
    k = _i64(0)
    _check(None, lib().grass_tree_segments(tree, C.byref(k), None, None), "grass_tree_segments")
    v, e = (_i64 * (k.value + 1))(), (_i64 * (k.value + 1))()
    _check(None, lib().grass_tree_segments(tree, None, v, e), "grass_tree_segments")
    return list(v), list(e)


def grass_densify_batch(ctx, forest, params: grass_params_t, h0, v0, nseg: int):
    """Returns (sparsifier, grass_sparsify_stats_t, per-graph rows of
    [lambda_min, lambda_max, theta, heat_max, added, embedded])."""
    out = _vp()
    st = grass_sparsify_stats_t()
    pg = (_d * (6 * nseg))()
    _check(ctx, lib().grass_densify_batch(ctx, forest, C.byref(params), _p(h0), _p(v0),
                                          C.byref(out), C.byref(st), pg), "grass_densify_batch")
    rows = [list(pg[6 * k:6 * k + 6]) for k in range(nseg)]
    return out.value, st, rows


def grass_pcg_solve_batch(ctx, S, b, x, tol: float, maxit: int, prec: int, inner_maxit: int,
                          nseg: int):
    """Returns (status, grass_solve_stats_t, iterations per graph, FP64
    relative residual per graph); NOT_CONVERGED is returned, not raised."""
    st = grass_solve_stats_t()
    its = (_i32 * nseg)()
    res = (_d * nseg)()
    s = _check(ctx, lib().grass_pcg_solve_batch(ctx, S, _p(b), _p(x), tol, maxit, prec,
                                                inner_maxit, C.byref(st), its, res),
               "grass_pcg_solve_batch", allow=(GRASS_ERR_NOT_CONVERGED,))
    return s, st, list(its), list(res)


def grass_autotune(ctx, tree, r: int, prec: int) -> tuple[list[int], float]:
    best = (_i64 * 3)()
    ms = _d(0.0)
    _check(ctx, lib().grass_autotune(ctx, tree, r, prec, best, C.byref(ms)), "grass_autotune")
    return list(best), ms.value
