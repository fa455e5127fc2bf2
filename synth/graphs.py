"""Seeded synthetic SDD matrices shaped like the paper's workloads.

Each generator returns a :class:`Graph` holding the full symmetric CSR of
``A = L_G + D`` (rows sorted by column, diagonal present, int64 row pointer,
int32 columns, float64 values).  ``L_G`` follows the Laplacian definition of
Section II-A (off-diagonal ``-w``, diagonal = weighted degree) and ``D`` is a
non-negative diagonal load (zero for a pure graph Laplacian).

The workloads stand in for the paper's power-grid, circuit/FEM and social
network matrices (Section V), which are not available here:

* 2D/3D grids with random conductances (circuit / thermal / FEM meshes);
* a Chung-Lu power-law graph, largest connected component only (data
  networks, Table VII);
* power-grid meshes with random long-range vias and pad loads (Tables I/II);
* rings with random chords (small uneven graphs for batching).

This module only builds inputs; it contains none of the sparsification
arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import rng


@dataclass
class Graph:
    name: str
    n: int
    rowptr: np.ndarray   # int64 [n+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def m(self) -> int:
        return (self.nnz - self.n) // 2


# --------------------------------------------------------------------------
# CSR assembly
# --------------------------------------------------------------------------

def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray, w: np.ndarray,
                   D: np.ndarray | float = 0.0) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Full symmetric CSR of L + diag(D) from an undirected edge list.

    Edges must be simple (no self loops, no duplicates).  Rows come out with
    ascending columns.
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    lo = np.minimum(u, v)
    hi = np.maximum(u, v)
    deg = np.bincount(lo, weights=w, minlength=n) + np.bincount(hi, weights=w, minlength=n)
    Dv = np.broadcast_to(np.asarray(D, dtype=np.float64), (n,))
    diag = deg + Dv
    ar = np.arange(n, dtype=np.int64)
    rows = np.concatenate([lo, hi, ar])
    cols = np.concatenate([hi, lo, ar])
    vals = np.concatenate([-w, -w, diag])
    key = rows * np.int64(n) + cols
    order = np.argsort(key, kind="stable")
    rows = rows[order]
    cols = cols[order].astype(np.int32)
    vals = vals[order]
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr, cols, vals


def _grid_edges(dims: tuple[int, ...]) -> tuple[np.ndarray, np.ndarray]:
    """Edges of a rectangular grid, in canonical (u asc, v asc) order.

    Vertex id = x + dims[0]*(y + dims[1]*z).  Each vertex links to its +1
    neighbour along each axis.
    """
    n = int(np.prod(dims))
    ids = np.arange(n, dtype=np.int64)
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    us, vs = [], []
    coord = []
    rem = ids.copy()
    for d in dims:
        coord.append(rem % d)
        rem //= d
    for ax, d in enumerate(dims):
        mask = coord[ax] < d - 1
        us.append(ids[mask])
        vs.append(ids[mask] + strides[ax])
    u = np.concatenate(us)
    v = np.concatenate(vs)
    order = np.lexsort((v, u))
    return u[order], v[order]


def grid(dims: tuple[int, ...], weights: np.ndarray | None = None, D=0.0,
         name: str | None = None) -> Graph:
    u, v = _grid_edges(dims)
    w = np.ones(u.shape[0]) if weights is None else weights
    n = int(np.prod(dims))
    rowptr, col, val = csr_from_edges(n, u, v, w, D)
    return Graph(name or "grid" + "x".join(map(str, dims)), n, rowptr, col, val,
                 {"dims": dims})


def n_grid_edges(dims: tuple[int, ...]) -> int:
    total = 0
    n = int(np.prod(dims))
    for d in dims:
        total += n // d * (d - 1)
    return total


# --------------------------------------------------------------------------
# Workload recipes
# --------------------------------------------------------------------------

def grid2d_uniform(nx: int, ny: int, seed: int, lo=1.0, hi=10.0, D=1e-3) -> Graph:
    """2D 5-point grid, w ~ U[lo, hi) in canonical edge order."""
    m = n_grid_edges((nx, ny))
    w = lo + (hi - lo) * rng.uniform(seed, rng.STREAM_WEIGHTS, m)
    g = grid((nx, ny), w, D, name=f"grid2d_{nx}x{ny}")
    g.meta.update(seed=seed, weights=f"U[{lo},{hi})", D=D)
    return g


def grid3d_loguniform(nx: int, ny: int, nz: int, seed: int, lo_exp=-2.0, hi_exp=2.0,
                      D=1e-3) -> Graph:
    """3D 7-point grid, w = 10^U(lo_exp, hi_exp) in canonical edge order."""
    m = n_grid_edges((nx, ny, nz))
    w = 10.0 ** (lo_exp + (hi_exp - lo_exp) * rng.uniform(seed, rng.STREAM_WEIGHTS, m))
    g = grid((nx, ny, nz), w, D, name=f"grid3d_{nx}x{ny}x{nz}")
    g.meta.update(seed=seed, weights=f"10^U({lo_exp},{hi_exp})", D=D)
    return g


def power_grid(k: int, seed: int, via_frac=0.01, via_w=100.0) -> Graph:
    """k x k power-grid mesh: wires w ~ U[0.1, 10], random long-range vias of
    weight via_w between non-adjacent node pairs, pad loads D ~ U[1e-4, 1e-2]."""
    n = k * k
    u, v = _grid_edges((k, k))
    w = 0.1 + 9.9 * rng.uniform(seed, rng.STREAM_WEIGHTS, u.shape[0])
    nv = int(round(via_frac * n))
    draws = rng.raw64(seed, rng.STREAM_EXTRA, 0, 2 * nv * 2)
    a = (draws[0::2] % np.uint64(n)).astype(np.int64)
    b = (draws[1::2] % np.uint64(n)).astype(np.int64)
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    ok = lo != hi
    dx = np.abs(lo % k - hi % k)
    dy = np.abs(lo // k - hi // k)
    ok &= (dx + dy) > 1                      # not a grid neighbour
    key = lo[ok] * n + hi[ok]
    _, first = np.unique(key, return_index=True)
    first = np.sort(first)[:nv]
    vu, vv = lo[ok][first], hi[ok][first]
    D = 1e-4 + (1e-2 - 1e-4) * rng.uniform(seed, rng.STREAM_PADS, n)
    uu = np.concatenate([u, vu])
    vvv = np.concatenate([v, vv])
    ww = np.concatenate([w, np.full(vu.shape[0], via_w)])
    rowptr, col, val = csr_from_edges(n, uu, vvv, ww, D)
    return Graph(f"powergrid_{k}x{k}", n, rowptr, col, val,
                 {"seed": seed, "vias": int(vu.shape[0]), "D": "U[1e-4,1e-2]"})


def ring_chords(n: int, seed: int, chord_frac=0.25, lo=1.0, hi=10.0, D=1e-3) -> Graph:
    """Ring 0-1-...-(n-1)-0 plus about chord_frac*n random chords."""
    ru = np.arange(n, dtype=np.int64)
    rv = (ru + 1) % n
    nc = int(chord_frac * n)
    draws = rng.raw64(seed, rng.STREAM_EXTRA, 0, 4 * nc)
    a = (draws[0::2] % np.uint64(n)).astype(np.int64)
    b = (draws[1::2] % np.uint64(n)).astype(np.int64)
    lo_, hi_ = np.minimum(a, b), np.maximum(a, b)
    ok = (hi_ - lo_ > 1) & ~((lo_ == 0) & (hi_ == n - 1))
    key = lo_[ok] * n + hi_[ok]
    _, first = np.unique(key, return_index=True)
    first = np.sort(first)[:nc]
    cu, cv = lo_[ok][first], hi_[ok][first]
    u = np.concatenate([np.minimum(ru, rv), cu])
    v = np.concatenate([np.maximum(ru, rv), cv])
    key = u * n + v
    order = np.argsort(key, kind="stable")
    u, v = u[order], v[order]
    w = lo + (hi - lo) * rng.uniform(seed, rng.STREAM_WEIGHTS, u.shape[0])
    rowptr, col, val = csr_from_edges(n, u, v, w, D)
    return Graph(f"ring{n}_chords", n, rowptr, col, val, {"seed": seed, "chords": int(cu.shape[0])})


def chung_lu(n: int, seed: int, mean_deg=10.0, beta=2.1) -> Graph:
    """Chung-Lu power-law graph with unit weights, largest component only.

    Expected degrees w_i ~ (i+1)^(-1/(beta-1)), scaled to the mean degree and
    capped at sqrt(sum w) so every pair probability stays <= 1.  About
    n*mean_deg/2 edges are drawn by endpoint sampling proportional to w; self
    loops and repeats are dropped.  Vertices of the largest connected
    component keep their relative order.
    """
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    alpha = 1.0 / (beta - 1.0)
    wt = (np.arange(n, dtype=np.float64) + 1.0) ** (-alpha)
    for _ in range(3):
        wt *= mean_deg * n / wt.sum()
        wt = np.minimum(wt, np.sqrt(wt.sum()))
    cdf = np.cumsum(wt)
    cdf /= cdf[-1]
    M = int(n * mean_deg / 2)
    uu = rng.uniform(seed, rng.STREAM_EXTRA, 2 * M)
    a = np.searchsorted(cdf, uu[0::2], side="right").astype(np.int64)
    b = np.searchsorted(cdf, uu[1::2], side="right").astype(np.int64)
    np.minimum(a, n - 1, out=a)
    np.minimum(b, n - 1, out=b)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    ok = lo != hi
    key = np.unique(lo[ok] * n + hi[ok])
    lo, hi = key // n, key % n
    adj = coo_matrix((np.ones(lo.shape[0]), (lo, hi)), shape=(n, n))
    ncomp, labels = connected_components(adj, directed=False)
    big = np.argmax(np.bincount(labels))
    keep = labels == big
    newid = np.full(n, -1, dtype=np.int64)
    newid[keep] = np.arange(int(keep.sum()))
    sel = keep[lo] & keep[hi]
    lo, hi = newid[lo[sel]], newid[hi[sel]]
    n2 = int(keep.sum())
    rowptr, col, val = csr_from_edges(n2, lo, hi, np.ones(lo.shape[0]), 0.0)
    return Graph(f"chunglu_{n}", n2, rowptr, col, val,
                 {"seed": seed, "n_sampled": n, "components": int(ncomp), "beta": beta,
                  "mean_deg": mean_deg})


# --------------------------------------------------------------------------
# The configurations of the benchmark suite
# --------------------------------------------------------------------------

def config_small_grid(seed: int = 1) -> Graph:
    """64x64 5-point grid, w ~ U[1,10), D = 1e-3 I (4096 nodes, 8064 edges)."""
    return grid2d_uniform(64, 64, seed)


def config_grid3d(side: int = 100, seed: int = 2) -> Graph:
    """side^3 7-point grid, log-uniform w in [1e-2, 1e2], D = 1e-3 I."""
    return grid3d_loguniform(side, side, side, seed)


def config_powerlaw(n: int = 4_000_000, seed: int = 3) -> Graph:
    return chung_lu(n, seed)


def config_powergrid(k: int, seed: int = 5) -> Graph:
    return power_grid(k, seed)


# --------------------------------------------------------------------------
# Batches of independent graphs
# --------------------------------------------------------------------------

def batch_union(gs: list[Graph]) -> tuple[Graph, list[int]]:
    """Block-diagonal union of several graphs: graph k occupies rows
    [off[k], off[k+1]) with its own column indices shifted by off[k]."""
    off = [0]
    for g in gs:
        off.append(off[-1] + g.n)
    rowptr = [np.zeros(1, dtype=np.int64)]
    cols, vals = [], []
    base = 0
    for g, o in zip(gs, off):
        rowptr.append(g.rowptr[1:] + base)
        cols.append(g.col.astype(np.int64) + o)
        vals.append(g.val)
        base += g.col.shape[0]
    rp = np.concatenate(rowptr)
    col = np.concatenate(cols).astype(np.int32)
    val = np.concatenate(vals)
    u = Graph(f"batch{len(gs)}", off[-1], rp, col, val, {"graphs": [g.name for g in gs]})
    return u, off


def config_batch(count: int = 256, seed: int = 7, side_lo: int = 32, side_hi: int = 512,
                 ring_lo: float = 1e3, ring_hi: float = 2e5) -> list[Graph]:
    """count/2 2D grids with side log-uniform in [side_lo, side_hi] and
    count/2 rings of n log-uniform in [ring_lo, ring_hi] with n/4 random
    chords; w ~ U[1,10), D = 1e-3 I.  Graph k uses seed + k."""
    u = rng.uniform(seed, rng.STREAM_EXTRA, count)
    gs = []
    for k in range(count):
        if k % 2 == 0:
            side = int(round(side_lo * (side_hi / side_lo) ** u[k]))
            gs.append(grid2d_uniform(side, side, seed + k))
        else:
            n = int(round(ring_lo * (ring_hi / ring_lo) ** u[k]))
            gs.append(ring_chords(n, seed + k))
    return gs


def hair_comb_edges(nx: int, ny: int) -> tuple[np.ndarray, np.ndarray]:
    """Vertex pairs (u < v) of the "hair-comb" spanning tree of the nx x ny
    grid (vertex id x + nx*y): the spine is row y = 0 and every column x is
    a tooth from y = 0 to y = ny - 1."""
    x = np.arange(nx - 1, dtype=np.int64)
    su, sv = x, x + 1
    xx, yy = np.meshgrid(np.arange(nx, dtype=np.int64), np.arange(ny - 1, dtype=np.int64),
                         indexing="xy")
    tu = (xx + nx * yy).ravel()
    return np.concatenate([su, tu]), np.concatenate([sv, tu + nx])
