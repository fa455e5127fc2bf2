// graph.cu -- validation of A = L_G + D and edge extraction (Sec. II-A,
// Eq. formula_laplacian): edges e = (u < v, w = -A(u,v)) numbered in
// row-major upper-triangle order, the off-diagonal adjacency of every row in
// CSR order with each entry's edge id, and D(p) = sum of row p.
#include "common.cuh"

namespace grass {

enum { FLAG_INVALID = 1, FLAG_NOT_SDD = 2 };

// Thread per row: structure checks, counts, D and weighted degree.  The row
// sum runs in CSR order, like the plain definition.
__global__ void k_rows(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col,
                       const double *val, int64_t *ucnt, int64_t *acnt, double *D, float *D32, double *degG,
                       int *flags) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t b = rowptr[p], e = rowptr[p + 1];
    if (b < 0 || e < b || e > nnz) {
        atomicOr(flags, FLAG_INVALID);
        ucnt[p] = acnt[p] = 0;
        return;
    }
    int64_t nu = 0, na = 0;
    double rowsum = 0.0, diag = 0.0, deg = 0.0;
    int32_t prev = -1;
    for (int64_t j = b; j < e; ++j) {
        int32_t q = col[j];
        double a = val[j];
        if (q < 0 || q >= n || q <= prev) atomicOr(flags, FLAG_INVALID);
        prev = q;
        rowsum += a;
        if (q == p) {
            diag = a;
            continue;
        }
        if (a > 0.0) atomicOr(flags, FLAG_INVALID);
        if (a == 0.0) continue;
        deg += -a;
        ++na;
        if (q > p) ++nu;
    }
    double Dp = rowsum;
    if (fabs(Dp) <= 1e-12 * fabs(diag)) Dp = 0.0;
    if (Dp < 0.0) atomicOr(flags, FLAG_NOT_SDD);
    D[p] = Dp;
    D32[p] = (float)Dp;
    degG[p] = deg;
    ucnt[p] = nu;
    acnt[p] = na;
}

__global__ void k_upper(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                        const int64_t *ebase, int32_t *eu, int32_t *ev, double *ew, float *ew32,
                        int32_t *entry_eid) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t e = ebase[p];
    for (int64_t j = rowptr[p]; j < rowptr[p + 1]; ++j) {
        int32_t q = col[j];
        double a = val[j];
        if (q > p && a < 0.0) {
            eu[e] = (int32_t)p;
            ev[e] = q;
            ew[e] = -a;
            ew32[e] = (float)(-a);
            entry_eid[j] = (int32_t)e;
            ++e;
        }
    }
}

__device__ inline int64_t find_in_row(const int64_t *rowptr, const int32_t *col, int64_t row,
                                      int32_t c) {
    int64_t lo = rowptr[row], hi = rowptr[row + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int32_t x = col[mid];
        if (x == c) return mid;
        if (x < c) lo = mid + 1;
        else hi = mid;
    }
    return -1;
}

__global__ void k_adj(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                      const int64_t *aoff, const int32_t *entry_eid, int32_t *adj_ptr,
                      int32_t *adj_col, int32_t *adj_eid, double *adj_w, float *adj_w32,
                      int *flags) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t k = aoff[p];
    adj_ptr[p] = (int32_t)k;
    if (p == n - 1) adj_ptr[n] = (int32_t)aoff[n];
    for (int64_t j = rowptr[p]; j < rowptr[p + 1]; ++j) {
        int32_t q = col[j];
        double a = val[j];
        if (q == p || a == 0.0) continue;
        int64_t t = find_in_row(rowptr, col, q, (int32_t)p);
        int32_t eid = -1;
        if (t < 0 || val[t] != a) {
            atomicOr(flags, FLAG_INVALID);     // asymmetric pattern or value
        } else {
            eid = q > p ? entry_eid[j] : entry_eid[t];
        }
        adj_col[k] = q;
        adj_eid[k] = eid;
        adj_w[k] = -a;
        adj_w32[k] = (float)(-a);
        ++k;
    }
}

// graph of every vertex, by binary search over the segment offsets
__global__ void k_seg_of(int64_t n, int64_t nseg, const int64_t *voff, int32_t *seg_of) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int64_t lo = 0, hi = nseg - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (voff[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    seg_of[v] = (int32_t)lo;
}

// a batch is block diagonal: no edge may join two graphs
__global__ void k_seg_check(int64_t m, const int32_t *eu, const int32_t *ev, const int32_t *seg_of,
                            int *flags) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m && seg_of[eu[e]] != seg_of[ev[e]]) atomicOr(flags, 4);
}

__global__ void k_gather_i64(int64_t cnt, const int64_t *idx, const int64_t *src, int64_t *dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) dst[i] = src[idx[i]];
}

static void check_flags(grass_ctx_t ctx, const char *stage) {
    int f = 0;
    d2h(ctx, &f, ctx->flags.p, sizeof(int));
    if (f & FLAG_INVALID) fail(GRASS_ERR_INVALID, std::string(stage) + ": malformed, positive or unmatched off-diagonal entry");
    if (f & FLAG_NOT_SDD) fail(GRASS_ERR_NOT_SDD, std::string(stage) + ": a row sum is negative (not diagonally dominant)");
}

void graph_extract(grass_ctx_t ctx, const grass_csr_t *A, GraphData &g) {
    int64_t n = A->n;
    if (n < 2) fail(GRASS_ERR_INVALID, "n must be >= 2");
    if (n >= (1LL << 31)) fail(GRASS_ERR_INVALID, "n must be < 2^31");
    if (!A->rowptr || !A->col || !A->val) fail(GRASS_ERR_INVALID, "null CSR pointer");
    int64_t ends[2];
    d2h(ctx, &ends[0], A->rowptr, sizeof(int64_t));
    d2h(ctx, &ends[1], A->rowptr + n, sizeof(int64_t));
    if (ends[0] != 0 || ends[1] != A->nnz) fail(GRASS_ERR_INVALID, "rowptr[0] != 0 or rowptr[n] != nnz");
    if (A->nnz >= (1LL << 31)) fail(GRASS_ERR_INVALID, "nnz must be < 2^31");
    memset_d(ctx, ctx->flags.p, 0, sizeof(int) * 4);

    g.n = n;
    g.D64.alloc(n);
    g.D32.alloc(n);
    g.degG.alloc(n);
    int64_t *ucnt = ctx->scr<int64_t>(SCR_TMP0, n + 1);
    int64_t *acnt = ctx->scr<int64_t>(SCR_TMP1, n + 1);
    int64_t *ebase = ctx->scr<int64_t>(SCR_TMP2, n + 1);
    int64_t *aoff = ctx->scr<int64_t>(SCR_TMP3, n + 1);
    launch(ctx, k_rows, cdiv(n, kBlock), kBlock, 0, n, A->nnz, A->rowptr, A->col, A->val, ucnt, acnt,
           g.D64.p, g.D32.p, g.degG.p, ctx->flags.p);
    check_flags(ctx, "validate");
    int64_t m = 0, na = 0;
    scan_i64(ctx, ucnt, ebase, n, &m);
    scan_i64(ctx, acnt, aoff, n, &na);
    if (na != 2 * m) fail(GRASS_ERR_INVALID, "off-diagonal pattern is not symmetric");
    if (m < n - g.nseg) fail(GRASS_ERR_DISCONNECTED, "fewer than n - (number of graphs) edges");
    g.m = m;
    g.eu.alloc(m);
    g.ev.alloc(m);
    g.ew64.alloc(m);
    g.ew32.alloc(m);
    int32_t *entry_eid = ctx->scr<int32_t>(SCR_Y, A->nnz + 1);
    launch(ctx, k_upper, cdiv(n, kBlock), kBlock, 0, n, A->rowptr, A->col, A->val,
           (const int64_t *)ebase, g.eu.p, g.ev.p, g.ew64.p, g.ew32.p, entry_eid);
    g.adj_ptr.alloc(n + 1);
    g.adj_col.alloc(2 * m);
    g.adj_eid.alloc(2 * m);
    g.adj_w64.alloc(2 * m);
    g.adj_w32.alloc(2 * m);
    launch(ctx, k_adj, cdiv(n, kBlock), kBlock, 0, n, A->rowptr, A->col, A->val,
           (const int64_t *)aoff, (const int32_t *)entry_eid, g.adj_ptr.p, g.adj_col.p,
           g.adj_eid.p, g.adj_w64.p, g.adj_w32.p, ctx->flags.p);
    check_flags(ctx, "symmetry");
    if (g.nseg > 1) {
        // vertex and edge ranges of every graph of the batch
        const int64_t G = g.nseg;
        DBuf<int64_t> &voff = g.seg_voff_d;
        DBuf<int64_t> tmp;
        voff.alloc(G + 1);
        tmp.alloc(G + 1);
        h2d(ctx, voff.p, g.seg_voff.data(), (G + 1) * sizeof(int64_t));
        g.seg_of.alloc(n);
        launch(ctx, k_seg_of, cdiv(n, kBlock), kBlock, 0, n, G, (const int64_t *)voff.p, g.seg_of.p);
        launch(ctx, k_seg_check, cdiv(m, kBlock), kBlock, 0, m, (const int32_t *)g.eu.p,
               (const int32_t *)g.ev.p, (const int32_t *)g.seg_of.p, ctx->flags.p);
        int f = 0;
        d2h(ctx, &f, ctx->flags.p, sizeof(int));
        if (f & 4) fail(GRASS_ERR_INVALID, "an edge joins two graphs of the batch");
        launch(ctx, k_gather_i64, cdiv(G + 1, kBlock), kBlock, 0, G + 1, (const int64_t *)voff.p,
               (const int64_t *)ebase, tmp.p);
        g.seg_eoff.resize(G + 1);
        d2h(ctx, g.seg_eoff.data(), tmp.p, (G + 1) * sizeof(int64_t));
    } else {
        g.seg_voff = {0, n};
        g.seg_eoff = {0, m};
    }
    // a pure graph Laplacian (no diagonal load anywhere)?
    unsigned long long *mb = (unsigned long long *)(ctx->scal.p + DS_MAX + 12);
    memset_d(ctx, mb, 0, sizeof(unsigned long long));
    max_abs_bits(ctx, GRASS_FP64, n, g.D64.p, mb);
    unsigned long long bits = 0;
    d2h(ctx, &bits, mb, sizeof(bits));
    g.lap_only = bits == 0;
    heavy_rows(ctx, n, 2 * m, g.adj_ptr.p, g.heavy);
}

}  // namespace grass
