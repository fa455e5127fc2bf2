/*
 * grass_oracle.c -- plain, slow, single-threaded FP64 reference of the GRASS
 * sparsify-and-solve path (Z. Feng, "GRASS: Graph Spectral Sparsification
 * Leveraging Scalable Spectral Perturbation Analysis", arXiv 1911.04382).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the GPU library is
 * compared against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may build, load or call it; the product path never does.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Every routine is the textbook form of the step it implements, written for a
 * reader to check against the paper by eye: no blocking, no fusion, no
 * reordering beyond what the definition states.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_ERR_INVALID 1
#define ORA_ERR_NOT_SDD 2
#define ORA_ERR_DISCONNECTED 3
#define ORA_ERR_NOT_CONVERGED 5

/* ------------------------------------------------------------------------
 * Section II-A, Eq. (formula_laplacian): L_G(p,q) = -w(p,q) for an edge,
 * L_G(p,p) = sum of incident weights.  The input is an SDD matrix
 * A = L_G + D stored as full symmetric CSR.  Edge e = (u < v, w = -A(u,v))
 * takes the rank of its upper-triangle entry in row-major order as its id;
 * D(p) = sum of row p (= A(p,p) - sum of incident weights).
 * Errors: malformed CSR, a positive or unmatched off-diagonal entry
 * (INVALID); D(p) < -1e-12 A(p,p) (NOT_SDD).  |D(p)| <= 1e-12 A(p,p) is
 * taken as exactly 0.
 * ---------------------------------------------------------------------- */
static int64_t find_col(const int64_t *rowptr, const int32_t *col, int64_t row, int32_t c)
{
    int64_t lo = rowptr[row], hi = rowptr[row + 1];   /* binary search, rows sorted */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] == c) return mid;
        if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    return -1;
}

int ora_extract(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                int64_t cap, int64_t *m_out, int32_t *eu, int32_t *ev, double *ew, double *D)
{
    if (n < 2 || rowptr[0] != 0) return ORA_ERR_INVALID;
    int64_t m = 0, lower = 0;
    for (int64_t p = 0; p < n; ++p) {
        if (rowptr[p + 1] < rowptr[p]) return ORA_ERR_INVALID;
        double rowsum = 0.0, diag = 0.0;
        int has_diag = 0;
        for (int64_t j = rowptr[p]; j < rowptr[p + 1]; ++j) {
            int32_t q = col[j];
            if (q < 0 || q >= n) return ORA_ERR_INVALID;
            if (j > rowptr[p] && col[j - 1] >= q) return ORA_ERR_INVALID; /* sorted, unique */
            rowsum += val[j];
            if (q == p) { diag = val[j]; has_diag = 1; continue; }
            if (val[j] > 0.0) return ORA_ERR_INVALID;
            if (val[j] == 0.0) continue;
            int64_t t = find_col(rowptr, col, q, (int32_t)p);
            if (t < 0 || val[t] != val[j]) return ORA_ERR_INVALID;   /* symmetric */
            if (q > p) {
                if (m >= cap) return ORA_ERR_INVALID;
                eu[m] = (int32_t)p; ev[m] = q; ew[m] = -val[j]; ++m;
            } else {
                ++lower;
            }
        }
        (void)has_diag;
        double Dp = rowsum;
        if (fabs(Dp) <= 1e-12 * fabs(diag)) Dp = 0.0;
        if (Dp < 0.0) return ORA_ERR_NOT_SDD;
        D[p] = Dp;
    }
    if (lower != m) return ORA_ERR_INVALID;
    *m_out = m;
    return ORA_OK;
}

/* ------------------------------------------------------------------------
 * Maximum-weight spanning tree by Kruskal's algorithm.  Edges are taken in
 * the strict total order (w descending, edge id ascending), so the tree is
 * unique.  Union-find with path halving and union by size.
 * Returns the number of connected components in *ncomp.
 * ---------------------------------------------------------------------- */
static int edge_before(const double *w, int64_t a, int64_t b)
{
    if (w[a] != w[b]) return w[a] > w[b];
    return a < b;
}

static void merge_sort_edges(int64_t *idx, int64_t *tmp, int64_t n, const double *w)
{
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) tmp[k++] = edge_before(w, idx[j], idx[i]) ? idx[j++] : idx[i++];
            while (i < mid) tmp[k++] = idx[i++];
            while (j < hi) tmp[k++] = idx[j++];
        }
        memcpy(idx, tmp, (size_t)n * sizeof(int64_t));
    }
}

static int64_t uf_find(int64_t *par, int64_t x)
{
    while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
    return x;
}

int ora_mst_kruskal(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                    const double *ew, uint8_t *in_tree, int64_t *ncomp)
{
    int64_t *idx = malloc((size_t)m * sizeof(int64_t));
    int64_t *tmp = malloc((size_t)m * sizeof(int64_t));
    int64_t *par = malloc((size_t)n * sizeof(int64_t));
    int64_t *sz = malloc((size_t)n * sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) { idx[e] = e; in_tree[e] = 0; }
    merge_sort_edges(idx, tmp, m, ew);
    for (int64_t v = 0; v < n; ++v) { par[v] = v; sz[v] = 1; }
    int64_t comps = n;
    for (int64_t k = 0; k < m && comps > 1; ++k) {
        int64_t e = idx[k];
        int64_t a = uf_find(par, eu[e]), b = uf_find(par, ev[e]);
        if (a == b) continue;
        if (sz[a] < sz[b]) { int64_t s = a; a = b; b = s; }
        par[b] = a; sz[a] += sz[b];
        in_tree[e] = 1;
        --comps;
    }
    *ncomp = comps;
    free(idx); free(tmp); free(par); free(sz);
    return comps == 1 ? ORA_OK : ORA_ERR_DISCONNECTED;
}

/* ------------------------------------------------------------------------
 * Orient the spanning tree at root rho by breadth-first search:
 * parent[v], pw[v] = weight of the edge v-parent(v), order = BFS order
 * (order[0] = rho).  Reversed BFS order lists every vertex after all of its
 * descendants, which is the leaf-first elimination order used below.
 * ---------------------------------------------------------------------- */
int ora_tree_orient(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                    const double *ew, const uint8_t *in_tree, int32_t rho,
                    int32_t *parent, double *pw, int32_t *order)
{
    int64_t *deg = calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e)
        if (in_tree[e]) { deg[eu[e] + 1]++; deg[ev[e] + 1]++; }
    for (int64_t v = 0; v < n; ++v) deg[v + 1] += deg[v];
    int64_t *fill = malloc((size_t)n * sizeof(int64_t));
    int32_t *adj = malloc((size_t)(deg[n] + 1) * sizeof(int32_t));
    double *adjw = malloc((size_t)(deg[n] + 1) * sizeof(double));
    for (int64_t v = 0; v < n; ++v) fill[v] = deg[v];
    for (int64_t e = 0; e < m; ++e)
        if (in_tree[e]) {
            adj[fill[eu[e]]] = ev[e]; adjw[fill[eu[e]]++] = ew[e];
            adj[fill[ev[e]]] = eu[e]; adjw[fill[ev[e]]++] = ew[e];
        }
    for (int64_t v = 0; v < n; ++v) parent[v] = -2;
    parent[rho] = -1; pw[rho] = 0.0;
    int64_t head = 0, tail = 0;
    order[tail++] = rho;
    while (head < tail) {
        int32_t v = order[head++];
        for (int64_t j = deg[v]; j < deg[v + 1]; ++j) {
            int32_t c = adj[j];
            if (parent[c] != -2) continue;
            parent[c] = v; pw[c] = adjw[j];
            order[tail++] = c;
        }
    }
    free(deg); free(fill); free(adj); free(adjw);
    return tail == n ? ORA_OK : ORA_ERR_DISCONNECTED;
}

/* ------------------------------------------------------------------------
 * Tree solve, Section III-H ("factorization of a tree-graph Laplacian ...
 * linear time") and Section III-F (a tiny diagonal added to one row makes
 * L_P invertible).
 *
 * D == NULL: X = grounded solution of L_T X = B at the root rho = order[0]
 * (X[rho] = 0).  This is the limit of adding delta > 0 to row rho: for any
 * B with zero column sums, delta * X[rho] = 1^T B = 0 whatever delta is.
 * D != NULL: X = (L_T + diag(D))^{-1} B; if the final pivot is not positive
 * (D identically zero) the root is grounded as above.
 *
 * Gaussian elimination of the tree matrix, leaves first (reversed BFS
 * order), pivot update d_p -= w^2 / d_v, then back substitution root first.
 * B and X are n x r row-major.
 * ---------------------------------------------------------------------- */
void ora_tree_solve(int64_t n, const int32_t *parent, const double *pw, const int32_t *order,
                    const double *D, int r, const double *B, double *X)
{
    double *d = malloc((size_t)n * sizeof(double));
    double *y = malloc((size_t)n * r * sizeof(double));
    for (int64_t v = 0; v < n; ++v) d[v] = D ? D[v] : 0.0;
    for (int64_t v = 0; v < n; ++v)
        if (parent[v] >= 0) { d[v] += pw[v]; d[parent[v]] += pw[v]; }
    memcpy(y, B, (size_t)n * r * sizeof(double));
    for (int64_t i = n - 1; i >= 1; --i) {
        int32_t v = order[i], p = parent[v];
        double mult = pw[v] / d[v];
        d[p] -= pw[v] * mult;
        for (int j = 0; j < r; ++j) y[(int64_t)p * r + j] += mult * y[(int64_t)v * r + j];
    }
    int32_t rho = order[0];
    for (int j = 0; j < r; ++j)
        X[(int64_t)rho * r + j] = (D && d[rho] > 0.0) ? y[(int64_t)rho * r + j] / d[rho] : 0.0;
    for (int64_t i = 1; i < n; ++i) {
        int32_t v = order[i], p = parent[v];
        for (int j = 0; j < r; ++j)
            X[(int64_t)v * r + j] = (y[(int64_t)v * r + j] + pw[v] * X[(int64_t)p * r + j]) / d[v];
    }
    free(d); free(y);
}

/* ------------------------------------------------------------------------
 * Y = L X for the Laplacian of the edges with mask[e] != 0 (all edges when
 * mask == NULL), from Eq. (formula_laplacian):
 *   (L x)_p = sum over edges (p,q) of w_pq (x_p - x_q).
 * X, Y are n x r row-major.
 * ---------------------------------------------------------------------- */
void ora_lap_apply(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev, const double *ew,
                   const uint8_t *mask, int r, const double *X, double *Y)
{
    memset(Y, 0, (size_t)n * r * sizeof(double));
    for (int64_t e = 0; e < m; ++e) {
        if (mask && !mask[e]) continue;
        int64_t a = eu[e], b = ev[e];
        for (int j = 0; j < r; ++j) {
            double f = ew[e] * (X[a * r + j] - X[b * r + j]);
            Y[a * r + j] += f;
            Y[b * r + j] -= f;
        }
    }
}

/* y = A x for the CSR matrix itself (A = L_G + D). */
void ora_csr_apply(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                   const double *x, double *y)
{
    for (int64_t p = 0; p < n; ++p) {
        double s = 0.0;
        for (int64_t j = rowptr[p]; j < rowptr[p + 1]; ++j) s += val[j] * x[col[j]];
        y[p] = s;
    }
}

/* ------------------------------------------------------------------------
 * Joule heat of every edge outside the sparsifier, Eqs. (formula_Joule),
 * (formula_pwr_iter5new) and (formula_pwr_iter6):
 *   heat_e = w_e * sum_j (H[p][j] - H[q][j])^2,  e = (p,q), in_s[e] == 0,
 * written compactly in increasing edge id.  Returns the number written.
 * ---------------------------------------------------------------------- */
int64_t ora_heat(int64_t m, const int32_t *eu, const int32_t *ev, const double *ew,
                 const uint8_t *in_s, int r, const double *H, double *heat)
{
    int64_t k = 0;
    for (int64_t e = 0; e < m; ++e) {
        if (in_s[e]) continue;
        int64_t a = eu[e], b = ev[e];
        double s = 0.0;
        for (int j = 0; j < r; ++j) {
            double dlt = H[a * r + j] - H[b * r + j];
            s += dlt * dlt;
        }
        heat[k++] = ew[e] * s;
    }
    return k;
}

/* Quadratic forms x^T L x of all edges and of the edges in S, per column:
 * qG[j] = sum_e w (dx)^2, qS[j] = same over in_s[e] != 0 (Eq. 2). */
void ora_quad_forms(int64_t m, const int32_t *eu, const int32_t *ev, const double *ew,
                    const uint8_t *in_s, int r, const double *X, double *qG, double *qS)
{
    for (int j = 0; j < r; ++j) { qG[j] = 0.0; qS[j] = 0.0; }
    for (int64_t e = 0; e < m; ++e) {
        int64_t a = eu[e], b = ev[e];
        for (int j = 0; j < r; ++j) {
            double dlt = X[a * r + j] - X[b * r + j];
            double h = ew[e] * dlt * dlt;
            qG[j] += h;
            if (in_s[e]) qS[j] += h;
        }
    }
}

/* ------------------------------------------------------------------------
 * Sparsifier solve X = (L_S + D)^{-1} Y, column by column.
 * in_s == NULL: S is the tree itself, solved directly.
 * Otherwise: conjugate gradients on L_S + D, x0 = 0, preconditioned by the
 * tree solve above (grounded at rho when D == NULL, in which case every
 * iterate keeps x[rho] = 0 and the result is the grounded solution).
 * Stops when ||r||_2 <= tol * ||y||_2 or after maxit updates.
 * iters[j] = updates done for column j.
 * ---------------------------------------------------------------------- */
static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static void lap_plus_diag(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                          const double *ew, const uint8_t *mask, const double *D,
                          const double *x, double *y)
{
    ora_lap_apply(n, m, eu, ev, ew, mask, 1, x, y);
    if (D) for (int64_t i = 0; i < n; ++i) y[i] += D[i] * x[i];
}

void ora_s_solve(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev, const double *ew,
                 const uint8_t *in_s, const int32_t *parent, const double *pw,
                 const int32_t *order, const double *D, int r, const double *Y, double *X,
                 double tol, int maxit, int32_t *iters)
{
    if (!in_s) {
        ora_tree_solve(n, parent, pw, order, D, r, Y, X);
        for (int j = 0; j < r; ++j) iters[j] = 0;
        return;
    }
    double *y = malloc((size_t)n * sizeof(double));
    double *x = malloc((size_t)n * sizeof(double));
    double *res = malloc((size_t)n * sizeof(double));
    double *z = malloc((size_t)n * sizeof(double));
    double *p = malloc((size_t)n * sizeof(double));
    double *q = malloc((size_t)n * sizeof(double));
    for (int j = 0; j < r; ++j) {
        for (int64_t i = 0; i < n; ++i) { y[i] = Y[i * r + j]; x[i] = 0.0; }
        if (!D) {
            /* L_S alone is singular: L_S^+ acts on the complement of the
             * all-ones vector, so the right-hand side is projected there
             * (its component along 1 is rounding, which CG cannot remove) */
            double mean = 0.0;
            for (int64_t i = 0; i < n; ++i) mean += y[i];
            mean /= (double)n;
            for (int64_t i = 0; i < n; ++i) y[i] -= mean;
        }
        for (int64_t i = 0; i < n; ++i) res[i] = y[i];
        double ynorm = sqrt(dot(n, y, y));
        ora_tree_solve(n, parent, pw, order, D, 1, res, z);
        memcpy(p, z, (size_t)n * sizeof(double));
        double rz = dot(n, res, z);
        int k = 0;
        for (; k < maxit; ++k) {
            if (sqrt(dot(n, res, res)) <= tol * ynorm) break;
            lap_plus_diag(n, m, eu, ev, ew, in_s, D, p, q);
            double pq = dot(n, p, q);
            if (pq <= 0.0) break;
            double alpha = rz / pq;
            for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; res[i] -= alpha * q[i]; }
            ora_tree_solve(n, parent, pw, order, D, 1, res, z);
            double rz_new = dot(n, res, z);
            double beta = rz_new / rz;
            rz = rz_new;
            for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        }
        iters[j] = k;
        for (int64_t i = 0; i < n; ++i) X[i * r + j] = x[i];
    }
    free(y); free(x); free(res); free(z); free(p); free(q);
}

/* ------------------------------------------------------------------------
 * PCG for A x = b, A = the input CSR (L_G + D), Section V-A: x0 = 0, stop at
 * ||b - A x||_2 <= tol ||b||_2.  Preconditioner M = L_S + D applied by
 * ora_s_solve (direct tree solve when in_s == NULL, else an inner CG with
 * inner_tol / inner_maxit, in which case the outer update uses the flexible
 * beta = r_new^T (z_new - z_old) / (r_old^T z_old)).
 * Returns NOT_CONVERGED if maxit updates were not enough; *iters, *relres
 * (recomputed as ||b - A x|| / ||b|| at exit) are always written.
 * ---------------------------------------------------------------------- */
int ora_pcg(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
            int64_t m, const int32_t *eu, const int32_t *ev, const double *ew,
            const uint8_t *in_s, const int32_t *parent, const double *pw, const int32_t *order,
            const double *D, const double *b, double *x, double tol, int maxit,
            double inner_tol, int inner_maxit, int32_t *iters, double *relres)
{
    double *res = malloc((size_t)n * sizeof(double));
    double *z = malloc((size_t)n * sizeof(double));
    double *zold = malloc((size_t)n * sizeof(double));
    double *p = malloc((size_t)n * sizeof(double));
    double *q = malloc((size_t)n * sizeof(double));
    int32_t it_in;
    int flexible = in_s != NULL;
    double bnorm = sqrt(dot(n, b, b));
    for (int64_t i = 0; i < n; ++i) { x[i] = 0.0; res[i] = b[i]; }
    ora_s_solve(n, m, eu, ev, ew, in_s, parent, pw, order, D, 1, res, z, inner_tol, inner_maxit, &it_in);
    memcpy(p, z, (size_t)n * sizeof(double));
    double rz = dot(n, res, z);
    int k = 0;
    for (; k < maxit; ++k) {
        if (sqrt(dot(n, res, res)) <= tol * bnorm) break;
        ora_csr_apply(n, rowptr, col, val, p, q);
        double alpha = rz / dot(n, p, q);
        for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; res[i] -= alpha * q[i]; }
        memcpy(zold, z, (size_t)n * sizeof(double));
        ora_s_solve(n, m, eu, ev, ew, in_s, parent, pw, order, D, 1, res, z, inner_tol, inner_maxit, &it_in);
        double rz_new = dot(n, res, z);
        double beta;
        if (flexible) {
            double s = 0.0;
            for (int64_t i = 0; i < n; ++i) s += res[i] * (z[i] - zold[i]);
            beta = s / rz;
        } else {
            beta = rz_new / rz;
        }
        rz = rz_new;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    ora_csr_apply(n, rowptr, col, val, x, q);
    for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
    *relres = sqrt(dot(n, q, q)) / bnorm;
    *iters = k;
    free(res); free(z); free(zold); free(p); free(q);
    return *relres <= tol ? ORA_OK : ORA_ERR_NOT_CONVERGED;
}
