"""CPU FP64 oracle of the GRASS sparsify-and-solve path (arXiv 1911.04382).

TEST INFRASTRUCTURE ONLY.  This package is the checker the GPU library is
compared against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the CUDA library (``paper_1911_04382_gb300``) and never
imports it.

The numeric kernels are plain single-threaded C (``grass_oracle.c``); the
orchestration below follows the paper's steps in the paper's order:

* Section II-A, Eq. (formula_laplacian): edges and the diagonal load D.
* Maximum-weight spanning tree (Kruskal, ties by edge id).
* Section III-F, Eqs. (formula_rand_vec), (formula_pwr_iter): t-step
  generalized power iteration h <- L_S^{-1} L_G h from a start block
  orthogonal to the all-ones vector, L_S made invertible by grounding one
  row (the limit of the paper's tiny diagonal on a random row).
* Eqs. (formula_pwr_iter5new), (formula_pwr_iter6): Joule heat of each
  off-sparsifier edge summed over the r vectors.
* Section IV-C: lambda_max by generalized power iterations (Rayleigh
  quotient), lambda_min by the node-degree ratio, Eq. (formula_courant-fischer-3).
* Eq. (formula_heatratio_final): threshold theta_sigma = (sigma^2 lmin/lmax)^(2t+1).
* Section IV-D: iterative densification.
* Section V-A: PCG on L_G + D preconditioned by the sparsifier.
* Section III-B: a low-stretch spanning tree (weight classes, shifted
  low-diameter decompositions with SplitMix64 shifts) and the total stretch
  st_T(G); pinned by ``tests/test_oracle_lsst.py``.

Pinned by ``tests/test_oracle_pins.py`` against dense linear algebra,
brute force and closed forms.  Unpinned parts (see the tests): the absolute
inner-CG iteration counts and the lambda_max value beyond the Courant-Fischer
bound.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "grass_oracle.c")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_NOT_SDD, ERR_DISCONNECTED, ERR_NOT_CONVERGED = 0, 1, 2, 3, 5


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"oracle {what}: status {status}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/liboracle.so (gcc, ISO C11,
    no FMA contraction so x86 and Arm builds round identically)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_i64, _i32, _f64, _u8 = C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_double), C.POINTER(C.c_uint8)


def _declare(L):
    L.ora_extract.argtypes = [C.c_int64, _i64, _i32, _f64, C.c_int64, _i64, _i32, _i32, _f64, _f64]
    L.ora_mst_kruskal.argtypes = [C.c_int64, C.c_int64, _i32, _i32, _f64, _u8, _i64]
    L.ora_tree_orient.argtypes = [C.c_int64, C.c_int64, _i32, _i32, _f64, _u8, C.c_int32, _i32, _f64, _i32]
    L.ora_tree_solve.argtypes = [C.c_int64, _i32, _f64, _i32, _f64, C.c_int, _f64, _f64]
    L.ora_tree_solve.restype = None
    L.ora_lap_apply.argtypes = [C.c_int64, C.c_int64, _i32, _i32, _f64, _u8, C.c_int, _f64, _f64]
    L.ora_lap_apply.restype = None
    L.ora_csr_apply.argtypes = [C.c_int64, _i64, _i32, _f64, _f64, _f64]
    L.ora_csr_apply.restype = None
    L.ora_heat.argtypes = [C.c_int64, _i32, _i32, _f64, _u8, C.c_int, _f64, _f64]
    L.ora_heat.restype = C.c_int64
    L.ora_quad_forms.argtypes = [C.c_int64, _i32, _i32, _f64, _u8, C.c_int, _f64, _f64, _f64]
    L.ora_quad_forms.restype = None
    L.ora_s_solve.argtypes = [C.c_int64, C.c_int64, _i32, _i32, _f64, _u8, _i32, _f64, _i32, _f64,
                              C.c_int, _f64, _f64, C.c_double, C.c_int, _i32]
    L.ora_s_solve.restype = None
    L.ora_pcg.argtypes = [C.c_int64, _i64, _i32, _f64, C.c_int64, _i32, _i32, _f64, _u8, _i32, _f64,
                          _i32, _f64, _f64, _f64, C.c_double, C.c_int, C.c_double, C.c_int, _i32, _f64]


def _p(a, t):
    if a is None:
        return None
    return a.ctypes.data_as(t)


# --------------------------------------------------------------------------
# Data held by the oracle
# --------------------------------------------------------------------------

@dataclass
class OGraph:
    """The oracle's view of A = L_G + D: the CSR plus the extracted edges."""
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    eu: np.ndarray = None
    ev: np.ndarray = None
    ew: np.ndarray = None
    D: np.ndarray = None

    @property
    def m(self) -> int:
        return int(self.eu.shape[0])


@dataclass
class OTree:
    in_tree: np.ndarray     # uint8[m]
    rho: int
    parent: np.ndarray      # int32[n]
    pw: np.ndarray          # float64[n]
    order: np.ndarray       # int32[n], BFS order from rho


@dataclass
class DensifyResult:
    in_s: np.ndarray
    rounds: int = 0
    added: list = field(default_factory=list)
    lmin: list = field(default_factory=list)
    lmax: list = field(default_factory=list)
    theta: list = field(default_factory=list)
    # per round: inner solves of the lambda_max estimate that reached inner_maxit
    capped: list = field(default_factory=list)
    stopped_similar: bool = False
    # per round, when densify(record=True): the heats of the off-S edges,
    # their ids, the threshold theta * heat_max and, with a cap, the heat of
    # the last edge the cap kept (None without one)
    trace: list = field(default_factory=list)


# --------------------------------------------------------------------------
# Steps
# --------------------------------------------------------------------------

def extract(n, rowptr, col, val) -> OGraph:
    """Edges (u<v, w) in id order and the diagonal load D (Eq. formula_laplacian)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    cap = max(1, (int(rowptr[-1]) - 0) // 2 + 1)
    eu = np.empty(cap, np.int32)
    ev = np.empty(cap, np.int32)
    ew = np.empty(cap, np.float64)
    D = np.empty(n, np.float64)
    m = C.c_int64(0)
    st = lib().ora_extract(n, _p(rowptr, _i64), _p(col, _i32), _p(val, _f64), cap, C.byref(m),
                           _p(eu, _i32), _p(ev, _i32), _p(ew, _f64), _p(D, _f64))
    if st != OK:
        raise OracleError(st, "extract")
    m = m.value
    return OGraph(n, rowptr, col, val, eu[:m].copy(), ev[:m].copy(), ew[:m].copy(), D)


def from_graph(g) -> OGraph:
    return extract(g.n, g.rowptr, g.col, g.val)


def mst(og: OGraph) -> np.ndarray:
    """Maximum-weight spanning tree, ties broken by smaller edge id."""
    in_tree = np.zeros(og.m, np.uint8)
    ncomp = C.c_int64(0)
    st = lib().ora_mst_kruskal(og.n, og.m, _p(og.eu, _i32), _p(og.ev, _i32), _p(og.ew, _f64),
                               _p(in_tree, _u8), C.byref(ncomp))
    if st != OK:
        raise OracleError(st, f"mst ({ncomp.value} components)")
    return in_tree


def orient(og: OGraph, in_tree: np.ndarray, rho: int = 0) -> OTree:
    parent = np.empty(og.n, np.int32)
    pw = np.empty(og.n, np.float64)
    order = np.empty(og.n, np.int32)
    st = lib().ora_tree_orient(og.n, og.m, _p(og.eu, _i32), _p(og.ev, _i32), _p(og.ew, _f64),
                               _p(in_tree, _u8), int(rho), _p(parent, _i32), _p(pw, _f64),
                               _p(order, _i32))
    if st != OK:
        raise OracleError(st, "orient")
    return OTree(in_tree.copy(), int(rho), parent, pw, order)


def build_tree(og: OGraph, rho: int = 0) -> OTree:
    return orient(og, mst(og), rho)


def _tree_solve_once(og, tree, B2, Dp, r):
    X = np.empty_like(B2)
    lib().ora_tree_solve(og.n, _p(tree.parent, _i32), _p(tree.pw, _f64), _p(tree.order, _i32),
                         _p(Dp, _f64), r, _p(B2, _f64), _p(X, _f64))
    return X


def tree_solve(og: OGraph, tree: OTree, B: np.ndarray, D: np.ndarray | None = None,
               refine: int = 2) -> np.ndarray:
    """(L_T + D)^{-1} B, or the solve grounded at tree.rho when D is None.

    The paper's operator is the exact inverse (Eq. formula_pwr_iter).  Leaf-
    first elimination forms pivots by subtraction and, on million-vertex
    trees with weights spread over decades, loses about 1e-8 relative
    accuracy; `refine` steps of residual correction (r = B - (L_T + D) X in
    FP64, X += solve(r)) bring the solve to full FP64 accuracy (one step
    already gives ~1e-14 on the 100^3 grid)."""
    B2 = np.ascontiguousarray(B, dtype=np.float64)
    r = 1 if B2.ndim == 1 else B2.shape[1]
    Dp = None if D is None else np.ascontiguousarray(D, dtype=np.float64)
    X = _tree_solve_once(og, tree, B2, Dp, r)
    for _ in range(refine):
        R = B2 - lap_apply(og, X, tree.in_tree)
        if Dp is not None:
            R -= (Dp[:, None] * X) if X.ndim == 2 else Dp * X
        else:
            R = R - R.mean(axis=0)      # the grounded system's right side sums to zero
        X = X + _tree_solve_once(og, tree, np.ascontiguousarray(R), Dp, r)
    return X


def lap_apply(og: OGraph, X: np.ndarray, mask: np.ndarray | None = None) -> np.ndarray:
    """L X for the graph Laplacian (no D) of all edges, or of mask[e] != 0."""
    X2 = np.ascontiguousarray(X, dtype=np.float64)
    r = 1 if X2.ndim == 1 else X2.shape[1]
    Y = np.empty_like(X2)
    lib().ora_lap_apply(og.n, og.m, _p(og.eu, _i32), _p(og.ev, _i32), _p(og.ew, _f64),
                        _p(mask, _u8), r, _p(X2, _f64), _p(Y, _f64))
    return Y


def csr_apply(og: OGraph, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    lib().ora_csr_apply(og.n, _p(og.rowptr, _i64), _p(og.col, _i32), _p(og.val, _f64),
                        _p(x, _f64), _p(y, _f64))
    return y


def heat(og: OGraph, in_s: np.ndarray, H: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Joule heat of every edge not in S, in increasing edge id (Eq. 5new/6)."""
    H2 = np.ascontiguousarray(H, dtype=np.float64)
    r = 1 if H2.ndim == 1 else H2.shape[1]
    off = np.flatnonzero(in_s == 0).astype(np.int64)
    out = np.empty(max(1, off.shape[0]), np.float64)
    k = lib().ora_heat(og.m, _p(og.eu, _i32), _p(og.ev, _i32), _p(og.ew, _f64), _p(in_s, _u8), r,
                       _p(H2, _f64), _p(out, _f64))
    assert k == off.shape[0]
    return out[:k], off


def quad_forms(og: OGraph, in_s: np.ndarray, X: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    X2 = np.ascontiguousarray(X, dtype=np.float64)
    r = 1 if X2.ndim == 1 else X2.shape[1]
    qG = np.empty(r)
    qS = np.empty(r)
    lib().ora_quad_forms(og.m, _p(og.eu, _i32), _p(og.ev, _i32), _p(og.ew, _f64), _p(in_s, _u8), r,
                         _p(X2, _f64), _p(qG, _f64), _p(qS, _f64))
    return qG, qS


def s_solve(og: OGraph, tree: OTree, in_s: np.ndarray | None, Y: np.ndarray,
            D: np.ndarray | None = None, tol: float = 1e-12, maxit: int = 1000):
    """(L_S + D)^{-1} Y: direct tree solve when in_s is None (S = tree), else
    CG on L_S + D preconditioned by the tree solve.  Returns (X, iters)."""
    Y2 = np.ascontiguousarray(Y, dtype=np.float64)
    r = 1 if Y2.ndim == 1 else Y2.shape[1]
    if in_s is None:
        return tree_solve(og, tree, Y2, D), np.zeros(r, np.int32)
    X = np.empty_like(Y2)
    it = np.zeros(r, np.int32)
    Dp = None if D is None else np.ascontiguousarray(D, dtype=np.float64)
    lib().ora_s_solve(og.n, og.m, _p(og.eu, _i32), _p(og.ev, _i32), _p(og.ew, _f64),
                      _p(in_s, _u8), _p(tree.parent, _i32), _p(tree.pw, _f64),
                      _p(tree.order, _i32), _p(Dp, _f64), r, _p(Y2, _f64), _p(X, _f64),
                      float(tol), int(maxit), _p(it, _i32))
    return X, it


def pow2_rescale(H: np.ndarray) -> np.ndarray:
    """Multiply by the power of two that puts max|H| in [1, 2): exact in
    binary floating point, the same factor for every column."""
    mx = float(np.max(np.abs(H)))
    if mx == 0.0 or not np.isfinite(mx):
        return H
    _, e = np.frexp(mx)
    return np.ldexp(H, -(int(e) - 1))


def _s_mask(tree: OTree, in_s: np.ndarray | None):
    """None when S is the tree itself (direct solve), else the edge mask."""
    if in_s is None or np.array_equal(in_s, tree.in_tree):
        return None
    return in_s


def embed(og: OGraph, tree: OTree, in_s: np.ndarray | None, h0: np.ndarray, t: int,
          inner_tol: float = 1e-12, inner_maxit: int = 1000) -> np.ndarray:
    """Eq. (formula_pwr_iter): h_t = (L_S^{-1} L_G)^t h_0, h_0 orthogonal to 1
    (Eq. formula_rand_vec), each step rescaled by a common power of two."""
    H = np.asarray(h0, dtype=np.float64)
    H = H - H.mean(axis=0, keepdims=True)
    mask = _s_mask(tree, in_s)
    for _ in range(t):
        Y = lap_apply(og, H)
        H, _ = s_solve(og, tree, mask, Y, None, inner_tol, inner_maxit)
        H = pow2_rescale(H)
    return H


def lambda_min_est(og: OGraph, in_s: np.ndarray) -> float:
    """Eq. (formula_courant-fischer-3): min over nodes of L_G(p,p)/L_S(p,p),
    the Laplacian diagonals (weighted degrees, D excluded)."""
    n = og.n
    dG = np.bincount(og.eu, og.ew, n) + np.bincount(og.ev, og.ew, n)
    s = in_s.astype(bool)
    dS = np.bincount(og.eu[s], og.ew[s], n) + np.bincount(og.ev[s], og.ew[s], n)
    return float(np.min(dG / dS))


def lambda_max_est(og: OGraph, tree: OTree, in_s: np.ndarray, v0: np.ndarray, iters: int,
                   inner_tol: float = 1e-12, inner_maxit: int = 1000) -> float:
    """Section IV-C-1: `iters` generalized power iterations from v0 (made
    orthogonal to 1), then the Rayleigh quotient v^T L_G v / v^T L_S v."""
    return lambda_max_est_checked(og, tree, in_s, v0, iters, inner_tol, inner_maxit)[0]


def lambda_max_est_checked(og: OGraph, tree: OTree, in_s: np.ndarray, v0: np.ndarray, iters: int,
                           inner_tol: float = 1e-12, inner_maxit: int = 1000,
                           stop_when_capped: bool = False):
    """lambda_max_est and the number of its inner CG solves that reached
    inner_maxit (0 when S is the tree: those solves are direct).  With
    stop_when_capped the power steps end after the first such solve and
    the quotient is taken on that step's vector."""
    v = np.asarray(v0, dtype=np.float64).reshape(-1, 1)
    v = v - v.mean()
    mask = _s_mask(tree, in_s)
    capped = 0
    for _ in range(iters):
        y = lap_apply(og, v)
        v, it = s_solve(og, tree, mask, y, None, inner_tol, inner_maxit)
        v = pow2_rescale(v)
        if mask is not None and int(np.max(it)) >= inner_maxit:
            capped += 1
            if stop_when_capped:
                break
    qG, qS = quad_forms(og, in_s, v)
    return float(qG[0] / qS[0]), capped


def theta_sigma(sigma2: float, lmin: float, lmax: float, t: int) -> float:
    """Eq. (formula_heatratio_final)."""
    return (sigma2 * lmin / lmax) ** (2 * t + 1)


def filter_edges(heat_vals: np.ndarray, off_eids: np.ndarray, theta: float, cap: int = 0) -> np.ndarray:
    """Keep off-tree edge e iff heat_e >= theta * heat_max.  With cap > 0,
    keep at most cap of them, by (heat descending, edge id ascending).
    Returns the kept edge ids in increasing order."""
    if heat_vals.shape[0] == 0:
        return np.zeros(0, np.int64)
    thr = theta * float(np.max(heat_vals))
    keep = np.flatnonzero(heat_vals >= thr)
    if cap > 0 and keep.shape[0] > cap:
        order = np.lexsort((off_eids[keep], -heat_vals[keep]))
        keep = np.sort(keep[order[:cap]])
    return off_eids[keep].astype(np.int64)


def similarity_check(og: OGraph, heat_vals: np.ndarray, off_eids: np.ndarray, theta: float,
                     cap: int = 0) -> np.ndarray:
    """Section IV-D step 6, "only add dissimilar edges", read as endpoint
    conflicts (the paper does not define similarity): the edges that pass
    the threshold theta * heat_max are visited in order of heat descending,
    smaller edge id first among equal heats; an edge is kept unless one of
    its endpoints is an endpoint of an edge kept before it; with cap > 0 the
    visit stops after cap kept edges.  Returns the kept ids in increasing
    order."""
    if heat_vals.shape[0] == 0:
        return np.zeros(0, np.int64)
    thr = theta * float(np.max(heat_vals))
    sel = np.flatnonzero(heat_vals >= thr)
    order = sel[np.lexsort((off_eids[sel], -heat_vals[sel]))]
    used = set()
    kept = []
    for i in order:
        e = int(off_eids[i])
        a, b = int(og.eu[e]), int(og.ev[e])
        if a in used or b in used:
            continue
        used.add(a)
        used.add(b)
        kept.append(e)
        if cap > 0 and len(kept) == cap:
            break
    return np.array(sorted(kept), dtype=np.int64)


def densify(og: OGraph, tree: OTree, h0s, v0s, sigma2: float, t: int, max_rounds: int,
            lmax_iters: int = 8, cap: int = 0, inner_tol: float = 1e-12,
            inner_maxit: int = 1000, record: bool = False,
            similarity: bool = False) -> DensifyResult:
    """Section IV-D: per round, (1) S updated, (2) lambda estimates,
    (3) stop when lmax/lmin <= sigma^2, (4) t-step power iteration with the
    round's r start vectors, (5) filter by theta_sigma, (6) with
    similarity=True keep only the edges similarity_check keeps (the paper
    leaves step 6 undefined; off by default), add the kept edges.

    An estimate whose inner solves stopped at inner_maxit is not trusted:
    it does not stop the loop, and theta_sigma takes the last trusted
    estimate instead (round 1's solves are direct tree solves, so there is
    always one).  Adding edges to S can only lower lambda_max(L_S^+ L_G),
    so that estimate is the best upper value at hand."""
    in_s = tree.in_tree.copy()
    res = DensifyResult(in_s)
    lmax_trusted = None
    for rd in range(max_rounds):
        lmin = lambda_min_est(og, in_s)
        # an estimate with a capped solve can neither stop the loop nor set
        # theta_sigma (below), so its power steps end at that solve
        lmax, capped = lambda_max_est_checked(og, tree, in_s, v0s[rd], lmax_iters, inner_tol,
                                              inner_maxit, stop_when_capped=True)
        res.lmin.append(lmin)
        res.lmax.append(lmax)
        res.capped.append(capped)
        # (3) a Rayleigh quotient bounds lambda_max from below only; one taken
        # after inner solves that stopped at their cap is not evidence of
        # similarity, so the stop test needs every solve to meet inner_tol
        if capped == 0 and lmax / lmin <= sigma2:
            res.stopped_similar = True
            break
        if capped == 0 or lmax_trusted is None:
            lmax_trusted = lmax
        H = embed(og, tree, in_s, h0s[rd], t, inner_tol, inner_maxit)
        hv, off = heat(og, in_s, H)
        th = theta_sigma(sigma2, lmin, lmax_trusted, t)
        res.theta.append(th)
        if similarity:
            acc = similarity_check(og, hv, off, th, cap)
        else:
            acc = filter_edges(hv, off, th, cap)
        if record:
            thr = th * float(np.max(hv)) if hv.shape[0] else 0.0
            kth = None
            if cap > 0 and acc.shape[0] == cap:
                kth = float(np.min(hv[np.searchsorted(off, acc)]))
            res.trace.append(dict(heat=hv, off=off, thr=thr, cap_heat=kth))
        res.rounds += 1
        res.added.append(int(acc.shape[0]))
        if acc.shape[0] == 0:
            break
        in_s = in_s.copy()
        in_s[acc] = 1
        res.in_s = in_s
    res.in_s = in_s
    return res


def pcg(og: OGraph, tree: OTree, in_s: np.ndarray | None, b: np.ndarray, tol: float,
        maxit: int = 1000, inner_tol: float = 1e-6, inner_maxit: int = 50):
    """Section V-A: PCG on A = L_G + D preconditioned by L_S + D.
    Returns (x, iterations, ||b - A x|| / ||b||, status)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty_like(b)
    it = C.c_int32(0)
    rel = C.c_double(0.0)
    mask = _s_mask(tree, in_s)
    # With D identically zero, L_S + D is a graph Laplacian: its solve is the
    # one grounded at the tree's root (the limit of Sec. III-F), not a division
    # by the root pivot, which elimination by subtraction leaves as a
    # rounding residue instead of zero.
    Dp = og.D if np.any(og.D != 0.0) else None
    st = lib().ora_pcg(og.n, _p(og.rowptr, _i64), _p(og.col, _i32), _p(og.val, _f64), og.m,
                       _p(og.eu, _i32), _p(og.ev, _i32), _p(og.ew, _f64), _p(mask, _u8),
                       _p(tree.parent, _i32), _p(tree.pw, _f64), _p(tree.order, _i32),
                       _p(Dp, _f64), _p(b, _f64), _p(x, _f64), float(tol), int(maxit),
                       float(inner_tol), int(inner_maxit), C.byref(it), C.byref(rel))
    return x, it.value, rel.value, st


def fiedler(og: OGraph, tree: OTree, in_s: np.ndarray | None, x0: np.ndarray, iters: int,
            tol: float, maxit: int = 5000, inner_tol: float = 1e-6, inner_maxit: int = 50):
    """Section V-F: spectral partitioning by a few inverse power iterations
    u <- A^{-1} u with A = L_G + D (for a graph Laplacian, D = 0: the
    Fiedler vector), u made orthogonal to the all-ones vector and of unit
    length before and after each solve, every solve by PCG preconditioned by
    the sparsifier (pcg); then the sign cut side = (u >= 0).  Returns
    (u, side, u^T L_G u, PCG iterations)."""
    x = np.asarray(x0, dtype=np.float64).copy()
    x -= x.mean()
    x /= np.linalg.norm(x)
    total = 0
    for _ in range(iters):
        y, it, rel, st = pcg(og, tree, in_s, x, tol, maxit, inner_tol, inner_maxit)
        total += it
        y -= y.mean()
        x = y / np.linalg.norm(y)
    qG, _ = quad_forms(og, np.ones(og.m, np.uint8), x)
    return x, (x >= 0).astype(np.uint8), float(qG[0]), total



# --------------------------------------------------------------------------
# Low-stretch spanning tree (Section III-B: the backbone the paper prefers to
# a maximum-weight tree).  Construction in the manner of Alon, Karp, Peleg
# and West: the edges fall into weight classes, heaviest first; within the
# edges of classes <= c the clusters are repeatedly split by a low-diameter
# decomposition (shifted breadth-first growth from cluster centres, after
# Miller, Peng and Xu) and contracted, the growth edges forming the tree.
# --------------------------------------------------------------------------

_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15
_LEVEL_MUL = 0xD1B54A32D192ED03
LSST_SHIFT_SCALE = 3    # shift = 3 x (leading zeros of a 64-bit draw)
LSST_SHIFT_CAP = 20     # on the leading zeros


def splitmix64(x: int) -> int:
    """Output of the SplitMix64 generator (Steele, Lea and Flood, 2014)
    whose state before the step is x: the state advances by the golden
    gamma 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds and a
    final xor-shift mix it."""
    z = (x + _GOLDEN) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def lsst_shift(seed: int, cls: int, level: int, x: int) -> int:
    """Integer shift of cluster x at (class, level): 3 times the number of
    leading zero bits (at most 20) of the SplitMix64 output for the state
    seed + (x + 1) G + (1000003 cls + level) H (mod 2^64), G the golden
    gamma and H = 0xD1B54A32D192ED03.  P(shift >= 3k) = 2^-k: a geometric
    stand-in for the exponential shifts of the decomposition."""
    st = (seed + (x + 1) * _GOLDEN + (cls * 1000003 + level) * _LEVEL_MUL) & _M64
    h = splitmix64(st)
    lz = 64 - h.bit_length()
    return LSST_SHIFT_SCALE * min(lz, LSST_SHIFT_CAP)


def lsst_classes(ew: np.ndarray) -> np.ndarray:
    """Weight class of each edge: emax - e, with e the binary exponent of w
    (w = f 2^e, 1/2 <= f < 1) and emax the largest; class 0 holds the
    heaviest edges and each class spans a factor of 2."""
    _, e = np.frexp(np.asarray(ew, dtype=np.float64))
    return (int(e.max()) - e).astype(np.int64)


def lsst_ldd(X, A, B, E, ew, start):
    """One low-diameter decomposition of the cluster graph whose vertices are
    the cluster ids X and whose edges are (A[k], B[k]) with graph edge ids
    E[k] (repeated pairs allowed).  start[x] is the round at which x would
    start its own cluster.  Rounds t = 0, 1, ...:
      1. an unclaimed cluster x adjacent to clusters claimed in round t-1
         joins, among their centres, the one with the smallest
         (start, centre id); it joins through the heaviest edge (smallest id
         on equal weight) to a neighbour claimed in round t-1 by that centre;
      2. every cluster still unclaimed whose start is t becomes a centre.
    Returns (centre, when, via): dicts over X of the centre, the round of
    the claim, and (non-centres only) the edge id it joined through."""
    nbr = {int(x): [] for x in X}
    for a, b, e in zip(A, B, E):
        nbr[int(a)].append((int(b), int(e)))
        nbr[int(b)].append((int(a), int(e)))
    centre = {int(x): -1 for x in X}
    when = {int(x): -1 for x in X}
    via = {}
    left = len(nbr)
    t = 0
    while left > 0:
        joins = {}
        for x, adj in nbr.items():
            if centre[x] >= 0:
                continue
            best = None
            for y, e in adj:
                if centre[y] < 0 or when[y] != t - 1:
                    continue
                c = centre[y]
                key = (start[c], c, -float(ew[e]), e)
                if best is None or key < best:
                    best = key
            if best is not None:
                joins[x] = best
        for x, key in joins.items():
            centre[x] = key[1]
            when[x] = t
            via[x] = key[3]
            left -= 1
        for x in nbr:
            if centre[x] < 0 and start[x] == t:
                centre[x] = x
                when[x] = t
                left -= 1
        t += 1
    return centre, when, via


def low_stretch_tree(og: OGraph, seed: int = 1) -> np.ndarray:
    """A low-stretch spanning tree of G (returns in_tree, uint8[m]).  For each
    weight class c = 0, 1, ... (lsst_classes) and level = 0, 1, ...: take
    the edges of classes <= c whose endpoints lie in different clusters
    (every vertex starts as its own cluster, named by its id); stop the
    class when there are none; else give each cluster x touched by them the
    shift s_x = lsst_shift(seed, c, level, x) and the start S - s_x (S the
    largest shift of the level), decompose (lsst_ldd), add every join edge
    to the tree and rename every cluster by its centre."""
    n, m = og.n, og.m
    cls = lsst_classes(og.ew)
    label = np.arange(n, dtype=np.int64)
    in_tree = np.zeros(m, np.uint8)
    for c in range(int(cls.max()) + 1):
        level = 0
        while True:
            a = label[og.eu]
            b = label[og.ev]
            act = np.flatnonzero((cls <= c) & (a != b))
            if act.shape[0] == 0:
                break
            X = np.unique(np.concatenate([a[act], b[act]]))
            shift = {int(x): lsst_shift(seed, c, level, int(x)) for x in X}
            S = max(shift.values())
            start = {x: S - s for x, s in shift.items()}
            centre, _, via = lsst_ldd(X, a[act], b[act], act, og.ew, start)
            for e in via.values():
                in_tree[e] = 1
            label = np.array([centre.get(int(l), int(l)) for l in label], dtype=np.int64)
            level += 1
    return in_tree


def total_stretch(og: OGraph, in_tree: np.ndarray) -> tuple[float, np.ndarray]:
    """Stretch of every edge, w_e times the resistance of the tree path
    between its endpoints (Section III-B; 1 for a tree edge), and their
    sum st_T(G), by walking the paths of the tree oriented from vertex 0."""
    tr = orient(og, in_tree, 0)
    depth = np.zeros(og.n, np.int64)
    dist = np.zeros(og.n)
    for v in tr.order[1:]:
        depth[v] = depth[tr.parent[v]] + 1
        dist[v] = dist[tr.parent[v]] + 1.0 / tr.pw[v]
    st = np.empty(og.m)
    for e in range(og.m):
        p, q = int(og.eu[e]), int(og.ev[e])
        a, b = p, q
        while depth[a] > depth[b]:
            a = tr.parent[a]
        while depth[b] > depth[a]:
            b = tr.parent[b]
        while a != b:
            a = tr.parent[a]
            b = tr.parent[b]
        st[e] = og.ew[e] * (dist[p] + dist[q] - 2.0 * dist[a])
    return float(st.sum()), st
