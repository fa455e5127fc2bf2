"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from
dense linear algebra on the edge list, brute force, or a closed form the
paper states.  A dropped term, a wrong sign or index, or a transposed operand
in the oracle fails at least one test below.
"""
import itertools

import numpy as np
import scipy.linalg
import pytest

import oracle
from synth import graphs, rng
from tests.helpers import dense_from_csr, dense_lap, gen_eigs, tiny_graph, tree_path


# ---------------------------------------------------------------- Eq. (formula_laplacian)

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_extract_reconstructs_matrix(seed):
    g = tiny_graph(9, 6, seed, D=0.0)
    og = oracle.from_graph(g)
    A = dense_from_csr(g)
    L = dense_lap(g.n, og.eu, og.ev, og.ew)
    assert np.allclose(L + np.diag(og.D), A, rtol=0, atol=1e-14)
    assert np.all(og.D == 0.0)                     # pure Laplacian: zero row sums
    assert np.all(og.eu < og.ev)
    # edge ids follow row-major upper-triangle order
    keys = og.eu.astype(np.int64) * g.n + og.ev
    assert np.all(np.diff(keys) > 0)


def test_extract_diagonal_load():
    g = graphs.grid2d_uniform(5, 4, seed=7, D=0.25)
    og = oracle.from_graph(g)
    assert np.allclose(og.D, 0.25, rtol=1e-13)
    assert og.m == graphs.n_grid_edges((5, 4))


def _csr_copy(g):
    return g.rowptr.copy(), g.col.copy(), g.val.copy()


def test_extract_errors():
    g = tiny_graph(6, 3, 4, D=0.1)
    rp, c, v = _csr_copy(g)
    off = np.flatnonzero(c != np.repeat(np.arange(g.n), np.diff(rp)))[0]
    v[off] = -v[off]                                 # positive off-diagonal
    with pytest.raises(oracle.OracleError) as ei:
        oracle.extract(g.n, rp, c, v)
    assert ei.value.status == oracle.ERR_INVALID
    rp, c, v = _csr_copy(g)
    v[off] *= 2.0                                    # asymmetric value
    with pytest.raises(oracle.OracleError) as ei:
        oracle.extract(g.n, rp, c, v)
    assert ei.value.status == oracle.ERR_INVALID
    rp, c, v = _csr_copy(g)
    diag = np.flatnonzero(c == np.repeat(np.arange(g.n), np.diff(rp)))[2]
    v[diag] -= 1.0                                   # D < 0
    with pytest.raises(oracle.OracleError) as ei:
        oracle.extract(g.n, rp, c, v)
    assert ei.value.status == oracle.ERR_NOT_SDD
    rp, c, v = _csr_copy(g)
    c[rp[1] - 1], c[rp[1] - 2] = c[rp[1] - 2], c[rp[1] - 1]   # unsorted row
    with pytest.raises(oracle.OracleError):
        oracle.extract(g.n, rp, c, v)


# ---------------------------------------------------------------- maximum spanning tree

def _acyclic(n, edges):
    par = list(range(n))

    def f(x):
        while par[x] != x:
            x = par[x]
        return x
    for a, b in edges:
        ra, rb = f(a), f(b)
        if ra == rb:
            return False
        par[ra] = rb
    return True


@pytest.mark.parametrize("seed", range(6))
def test_mst_matches_brute_force(seed):
    """With weight ties (integer weights), the unique maximum tree under the
    order (w desc, id asc) is the lexicographically best spanning tree."""
    g = tiny_graph(7, 5, 100 + seed, integer_weights=True)
    og = oracle.from_graph(g)
    keyed = [(-og.ew[e], e) for e in range(og.m)]
    best = None
    for comb in itertools.combinations(range(og.m), g.n - 1):
        if not _acyclic(g.n, [(og.eu[e], og.ev[e]) for e in comb]):
            continue
        sig = sorted(keyed[e] for e in comb)
        if best is None or sig < best[0]:
            best = (sig, set(comb))
    assert set(np.flatnonzero(oracle.mst(og))) == best[1]


def test_mst_cycle_property_small_grid():
    """Every off-tree edge comes after every tree edge on its tree path."""
    g = graphs.grid2d_uniform(12, 10, seed=5)
    og = oracle.from_graph(g)
    in_tree = oracle.mst(og)
    assert in_tree.sum() == g.n - 1

    def key(e):
        return (-og.ew[e], e)
    for e in np.flatnonzero(in_tree == 0):
        path = tree_path(g.n, og.eu, og.ev, in_tree, int(og.eu[e]), int(og.ev[e]))
        assert all(key(f) < key(e) for f in path)


def test_disconnected_graph_reports_components():
    u = np.array([0, 2])
    v = np.array([1, 3])
    rp, c, val = graphs.csr_from_edges(4, u, v, np.ones(2))
    og = oracle.extract(4, rp, c, val)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.mst(og)
    assert ei.value.status == oracle.ERR_DISCONNECTED


# ---------------------------------------------------------------- tree solve

@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_tree_solve_matches_pinv(seed):
    g = tiny_graph(11, 7, 200 + seed)
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og, rho=seed % g.n)
    LT = dense_lap(g.n, og.eu, og.ev, og.ew, tree.in_tree)
    B = rng.gaussian_block(seed, 5, g.n, 3)
    B -= B.mean(axis=0)
    X = oracle.tree_solve(og, tree, B)
    assert np.all(X[tree.rho] == 0.0)                       # grounded row
    ref = scipy.linalg.pinv(LT) @ B
    Xc = X - X.mean(axis=0)
    assert np.allclose(Xc, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_tree_solve_with_diagonal_matches_dense():
    g = tiny_graph(13, 4, 9)
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og, rho=3)
    LT = dense_lap(g.n, og.eu, og.ev, og.ew, tree.in_tree)
    D = 1e-3 + rng.uniform(9, 6, g.n)
    B = rng.gaussian_block(9, 7, g.n, 2)
    X = oracle.tree_solve(og, tree, B, D)
    ref = np.linalg.solve(LT + np.diag(D), B)
    assert np.allclose(X, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_tree_effective_resistance_is_path_sum():
    """Eq. (formula_Reff) for a tree: e_pq^T L_T^+ e_pq = sum of 1/w on the path."""
    g = tiny_graph(10, 8, 31)
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og)
    for p in range(g.n):
        for q in range(p + 1, g.n):
            b = np.zeros(g.n)
            b[p], b[q] = 1.0, -1.0
            x = oracle.tree_solve(og, tree, b.reshape(-1, 1))[:, 0]
            path = tree_path(g.n, og.eu, og.ev, tree.in_tree, p, q)
            assert np.isclose(x[p] - x[q], sum(1.0 / og.ew[e] for e in path), rtol=1e-12)


def test_trace_equals_total_stretch():
    """Eq. (formula_trace): Tr(L_T^+ L_G) = st_T(G) (Eqs. stretch_graph/edge)."""
    g = tiny_graph(12, 10, 41)
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og)
    LG = dense_lap(g.n, og.eu, og.ev, og.ew)
    LT = dense_lap(g.n, og.eu, og.ev, og.ew, tree.in_tree)
    st = 0.0
    for e in range(og.m):
        path = tree_path(g.n, og.eu, og.ev, tree.in_tree, int(og.eu[e]), int(og.ev[e]))
        st += og.ew[e] * sum(1.0 / og.ew[f] for f in path)
    assert np.isclose(np.trace(scipy.linalg.pinv(LT) @ LG), st, rtol=1e-10)
    # and through the oracle's own solve: sum_e w_e R_eff(e)
    tot = 0.0
    for e in range(og.m):
        b = np.zeros((g.n, 1))
        b[og.eu[e]], b[og.ev[e]] = 1.0, -1.0
        x = oracle.tree_solve(og, tree, b)
        tot += og.ew[e] * (x[og.eu[e], 0] - x[og.ev[e], 0])
    assert np.isclose(tot, st, rtol=1e-12)


def test_root_choice_does_not_change_heat():
    g = graphs.grid2d_uniform(9, 7, seed=3)
    og = oracle.from_graph(g)
    h0 = rng.gaussian_block(3, rng.STREAM_H0, g.n, 4)
    heats = []
    for rho in (0, 17, g.n - 1):
        tree = oracle.build_tree(og, rho)
        H = oracle.embed(og, tree, None, h0, 2)
        hv, _ = oracle.heat(og, tree.in_tree, H)
        heats.append(hv / hv.max())
    assert np.allclose(heats[0], heats[1], rtol=0, atol=1e-12)
    assert np.allclose(heats[0], heats[2], rtol=0, atol=1e-12)


# ---------------------------------------------------------------- Laplacian products

def test_lap_apply_matches_dense():
    g = tiny_graph(14, 9, 51, D=0.3)
    og = oracle.from_graph(g)
    X = rng.gaussian_block(51, 8, g.n, 5)
    LG = dense_lap(g.n, og.eu, og.ev, og.ew)
    assert np.allclose(oracle.lap_apply(og, X), LG @ X, rtol=0, atol=1e-13)
    mask = (np.arange(og.m) % 3 == 0).astype(np.uint8)
    LS = dense_lap(g.n, og.eu, og.ev, og.ew, mask)
    assert np.allclose(oracle.lap_apply(og, X, mask), LS @ X, rtol=0, atol=1e-13)
    A = dense_from_csr(g)
    x = X[:, 0].copy()
    assert np.allclose(oracle.csr_apply(og, x), A @ x, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- power iteration, heat

def _dense_embed(LG, LS, h0, t):
    P = scipy.linalg.pinv(LS) @ LG
    H = h0 - h0.mean(axis=0)
    for _ in range(t):
        H = P @ H
    return H


def _heat_dense(og, in_s, H):
    off = np.flatnonzero(in_s == 0)
    d = H[og.eu[off]] - H[og.ev[off]]
    return og.ew[off] * np.sum(d * d, axis=1)


@pytest.mark.parametrize("with_extra", [False, True])
def test_embed_and_heat_match_dense(with_extra):
    g = graphs.grid2d_uniform(6, 5, seed=8)
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og)
    in_s = tree.in_tree.copy()
    if with_extra:
        off = np.flatnonzero(in_s == 0)
        in_s[off[::3]] = 1
    LG = dense_lap(g.n, og.eu, og.ev, og.ew)
    LS = dense_lap(g.n, og.eu, og.ev, og.ew, in_s)
    h0 = rng.gaussian_block(8, rng.STREAM_H0, g.n, 4)
    for t in (1, 2, 3):
        H = oracle.embed(og, tree, in_s, h0, t, inner_tol=1e-14, inner_maxit=500)
        ref = _dense_embed(LG, LS, h0, t)
        hv, off = oracle.heat(og, in_s, H)
        hr = _heat_dense(og, in_s, ref)
        assert np.allclose(hv / hv.max(), hr / hr.max(), rtol=0, atol=1e-10)
        # same vector up to an additive constant and a common power of two
        s = np.abs(H - H.mean(0)).max() / np.abs(ref - ref.mean(0)).max()
        assert np.allclose((H - H.mean(0)) / s, ref - ref.mean(0), rtol=0,
                           atol=1e-9 * np.abs(ref).max())
        assert np.isclose(s, 2.0 ** np.round(np.log2(s)), rtol=1e-9)


def test_heat_sum_is_quadratic_form_of_missing_edges():
    """Eq. (formula_pwr_iter5new): sum over edges not in S of the heat equals
    h^T (L_G - L_S) h, summed over the r vectors (Eq. pwr_iter6)."""
    g = tiny_graph(15, 12, 61)
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og)
    H = oracle.embed(og, tree, None, rng.gaussian_block(61, 9, g.n, 3), 2)
    hv, _ = oracle.heat(og, tree.in_tree, H)
    dL = dense_lap(g.n, og.eu, og.ev, og.ew) - dense_lap(g.n, og.eu, og.ev, og.ew, tree.in_tree)
    assert np.isclose(hv.sum(), np.trace(H.T @ dL @ H), rtol=1e-12)


def test_adding_all_heated_edges_gives_unit_spectrum():
    """P. III-F: adding every off-tree edge with nonzero heat brings all
    generalized eigenvalues to 1."""
    g = tiny_graph(10, 8, 71)
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og)
    H = oracle.embed(og, tree, None, rng.gaussian_block(71, 9, g.n, 2), 2)
    hv, off = oracle.heat(og, tree.in_tree, H)
    in_s = tree.in_tree.copy()
    in_s[off[hv > 0]] = 1
    lam = gen_eigs(dense_lap(g.n, og.eu, og.ev, og.ew), dense_lap(g.n, og.eu, og.ev, og.ew, in_s))
    assert np.allclose(lam, 1.0, atol=1e-10)


def _cycle(n, w_off):
    u = np.arange(n - 1)
    v = u + 1
    w = 1.0 + (np.arange(n - 1) % 3)
    u = np.append(u, 0)
    v = np.append(v, n - 1)
    w = np.append(w, w_off)
    order = np.lexsort((v, u))
    rp, c, val = graphs.csr_from_edges(n, u[order], v[order], w[order])
    return graphs.Graph("cycle", n, rp, c, val)


def test_cycle_dominant_eigenvalue_is_one_plus_stretch():
    """Sections III-F/III-G on a cycle: tree = path, one off-tree edge e.
    L_T^+ L_G has the single non-unit eigenvalue 1 + st_T(e) (Eq. eigfix3,
    R_eff = path sum), adding e fixes it to 1 (Eq. rank_one_update4)."""
    n, w_off = 12, 0.7
    g = _cycle(n, w_off)
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og)
    e = int(np.flatnonzero(tree.in_tree == 0)[0])
    path = tree_path(n, og.eu, og.ev, tree.in_tree, int(og.eu[e]), int(og.ev[e]))
    st = og.ew[e] * sum(1.0 / og.ew[f] for f in path)
    LG = dense_lap(n, og.eu, og.ev, og.ew)
    LT = dense_lap(n, og.eu, og.ev, og.ew, tree.in_tree)
    lam = gen_eigs(LG, LT)
    assert np.isclose(lam.max(), 1.0 + st, rtol=1e-12)
    assert np.allclose(np.sort(lam)[:-1], 1.0, atol=1e-12)
    # the power-iteration estimate converges to it (one non-unit eigenvalue)
    lm = oracle.lambda_max_est(og, tree, tree.in_tree, rng.normal(5, 1, n), 20)
    assert np.isclose(lm, 1.0 + st, rtol=1e-10)
    # rank-one update: lambda' = lambda / (1 + w gamma^2) = 1
    gamma2 = sum(1.0 / og.ew[f] for f in path)
    assert np.isclose((1 + st) / (1 + og.ew[e] * gamma2), 1.0, rtol=1e-14)
    in_s = tree.in_tree.copy()
    in_s[e] = 1
    assert np.allclose(gen_eigs(LG, dense_lap(n, og.eu, og.ev, og.ew, in_s)), 1.0, atol=1e-10)


# ---------------------------------------------------------------- eigenvalue estimates

@pytest.mark.parametrize("seed", [3, 4])
def test_lambda_estimates_bound_the_true_extremes(seed):
    g = graphs.grid2d_uniform(8, 7, seed=seed)
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og)
    in_s = tree.in_tree.copy()
    off = np.flatnonzero(in_s == 0)
    in_s[off[::4]] = 1
    LG = dense_lap(g.n, og.eu, og.ev, og.ew)
    for mask in (tree.in_tree, in_s):
        lam = gen_eigs(LG, dense_lap(g.n, og.eu, og.ev, og.ew, mask))
        lmax = oracle.lambda_max_est(og, tree, mask, rng.normal(seed, 3, g.n), 8,
                                     inner_tol=1e-14, inner_maxit=500)
        lmin = oracle.lambda_min_est(og, mask)
        assert lmax <= lam.max() * (1 + 1e-10)       # Courant-Fischer (Eq. courant-fischer-max)
        assert lmax >= 0.5 * lam.max()               # sanity: power iteration is close
        assert lmin >= lam.min() * (1 - 1e-10)       # Eq. (courant-fischer-3): upper bound
        assert lam.min() >= 1.0 - 1e-10              # unscaled subgraph: lambda_min >= 1


# ---------------------------------------------------------------- filter

def test_threshold_formula():
    # Eq. (formula_heatratio_final) with t = 2: exponent 5
    assert oracle.theta_sigma(100.0, 1.5, 6000.0, 2) == pytest.approx((150.0 / 6000.0) ** 5, rel=1e-15)


def test_filter_threshold_and_cap():
    hv = np.array([5.0, 1.0, 5.0, 0.2, 3.0, 5.0, 0.0])
    ids = np.array([10, 11, 12, 13, 14, 15, 16])
    assert list(oracle.filter_edges(hv, ids, 0.5)) == [10, 12, 14, 15]
    assert list(oracle.filter_edges(hv, ids, 0.5, cap=2)) == [10, 12]       # ties -> smaller id
    assert list(oracle.filter_edges(hv, ids, 0.5, cap=3)) == [10, 12, 15]
    assert list(oracle.filter_edges(hv, ids, 0.0)) == list(ids)
    assert list(oracle.filter_edges(hv, ids, 1.0)) == [10, 12, 15]


# ---------------------------------------------------------------- densification

def test_densify_reduces_condition_number():
    g = graphs.grid2d_uniform(10, 10, seed=1)
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og)
    h0s = [rng.gaussian_block(1, rng.STREAM_H0 + k, g.n, 8) for k in range(3)]
    v0s = [rng.normal(1, rng.STREAM_V0 + k, g.n) for k in range(3)]
    LG = dense_lap(g.n, og.eu, og.ev, og.ew)
    k0 = gen_eigs(LG, dense_lap(g.n, og.eu, og.ev, og.ew, tree.in_tree))
    res = oracle.densify(og, tree, h0s, v0s, sigma2=20.0, t=2, max_rounds=3, cap=8,
                         inner_tol=1e-13, inner_maxit=500)
    lam = gen_eigs(LG, dense_lap(g.n, og.eu, og.ev, og.ew, res.in_s))
    assert res.rounds >= 1 and sum(res.added) == int(res.in_s.sum()) - (g.n - 1)
    assert lam.max() / lam.min() < k0.max() / k0.min()
    assert all(a <= 8 for a in res.added)
    # the estimates of round 1 bound the tree's true extremes
    assert res.lmax[0] <= k0.max() * (1 + 1e-10)
    assert res.lmin[0] >= k0.min() * (1 - 1e-10)


def test_densify_stops_when_similar():
    g = graphs.grid2d_uniform(6, 6, seed=2)
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og)
    h0s = [rng.gaussian_block(2, rng.STREAM_H0, g.n, 4)]
    v0s = [rng.normal(2, rng.STREAM_V0, g.n)]
    res = oracle.densify(og, tree, h0s, v0s, sigma2=1e9, t=2, max_rounds=1)
    assert res.stopped_similar and res.rounds == 0


def test_densify_untrusted_estimate_keeps_filtering():
    """One inner CG iteration: from round 2 on, the lambda_max estimate comes
    from capped solves.  Round 2's estimate (about 1.6) claims similarity
    under sigma^2 = 5 while the dense generalized eigensolve puts the
    sparsifier's kappa near 17; theta_sigma from that estimate exceeds 1 and
    would reject every edge.  The loop neither stops nor takes that theta:
    it filters with the last trusted estimate, which can only be an upper
    value (lambda_max falls as edges are added), and each round's edges
    lower the true kappa."""
    g = graphs.grid3d_loguniform(8, 8, 8, seed=2)
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og)
    R, sigma2, t = 3, 5.0, 2
    h0s = [rng.gaussian_block(9, rng.STREAM_H0 + k, g.n, 8) for k in range(R)]
    v0s = [rng.normal(9, rng.STREAM_V0 + k, g.n) for k in range(R)]
    LG = dense_lap(g.n, og.eu, og.ev, og.ew)
    res = oracle.densify(og, tree, h0s, v0s, sigma2, t, R, 8, cap=30, inner_tol=1e-13,
                         inner_maxit=1)
    # the estimate ends at its first capped solve
    assert res.capped == [0, 1, 1]
    assert res.rounds == R and res.added == [30, 30, 30]
    kappas = []
    for k in range(R + 1):
        in_s = tree.in_tree if k == 0 else oracle.densify(
            og, tree, h0s, v0s, sigma2, t, k, 8, cap=30, inner_tol=1e-13, inner_maxit=1).in_s
        lam = gen_eigs(LG, dense_lap(g.n, og.eu, og.ev, og.ew, in_s))
        kappas.append(lam.max() / lam.min())
        if 0 < k < R:
            # round k+1's estimate is far below the truth and claims similarity
            assert res.lmax[k] / res.lmin[k] <= sigma2 < kappas[k]
            assert oracle.theta_sigma(sigma2, res.lmin[k], res.lmax[k], t) > 1.0
            # the theta used is no stricter than the one the exact lambda_max gives
            exact = (sigma2 * res.lmin[k] / lam.max()) ** (2 * t + 1)
            assert res.theta[k] <= exact
    assert all(a > b for a, b in zip(kappas, kappas[1:]))


# ---------------------------------------------------------------- PCG

def test_pcg_matches_dense_solve():
    g = graphs.grid2d_uniform(9, 8, seed=4, D=1e-3)
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og)
    b = rng.normal(4, rng.STREAM_RHS, g.n)
    A = dense_from_csr(g)
    ref = np.linalg.solve(A, b)
    x, it, rel, st = oracle.pcg(og, tree, None, b, 1e-10, maxit=2000)
    assert st == 0 and rel <= 1e-10
    assert np.allclose(x, ref, rtol=0, atol=1e-8 * np.abs(ref).max())
    in_s = tree.in_tree.copy()
    in_s[np.flatnonzero(in_s == 0)[::2]] = 1
    x2, it2, rel2, st2 = oracle.pcg(og, tree, in_s, b, 1e-10, maxit=2000, inner_tol=1e-12,
                                    inner_maxit=500)
    assert st2 == 0 and np.allclose(x2, ref, rtol=0, atol=1e-6 * np.abs(ref).max())
    assert it2 < it


def test_pcg_on_a_tree_converges_in_one_iteration():
    g = tiny_graph(20, 0, 5, D=0.01)          # a spanning path only
    og = oracle.from_graph(g)
    tree = oracle.build_tree(og)
    b = rng.normal(5, 1, g.n)
    x, it, rel, st = oracle.pcg(og, tree, None, b, 1e-12, maxit=10)
    assert st == 0 and it == 1 and rel < 1e-12


def test_pow2_rescale_is_exact():
    H = rng.gaussian_block(1, 1, 50, 3) * 1e7
    R = oracle.pow2_rescale(H)
    assert 1.0 <= np.abs(R).max() < 2.0
    f = R[0, 0] / H[0, 0]
    assert np.all(R == H * f) and f == 2.0 ** np.round(np.log2(f))
