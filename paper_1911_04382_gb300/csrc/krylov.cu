// krylov.cu -- sparsifier solves (tree solve or tree-preconditioned CG over
// r columns) and the PCG solver of A = L_G + D (Sec. V-A).
#include <cmath>

#include "common.cuh"

namespace grass {

// per-column CG scalars in the device scalar area
enum { CG_RZ = 0, CG_RR, CG_YY, CG_PQ, CG_ALPHA, CG_RZN, CG_ACT, CG_BROKEN, CG_IT, CG_NACT, CG_N };

__global__ void k_cg_init_scalars(int r, double *cg) {
    int j = threadIdx.x;
    if (j < r) {
        cg[CG_YY * 32 + j] = cg[CG_RR * 32 + j];
        cg[CG_BROKEN * 32 + j] = 0.0;
        cg[CG_IT * 32 + j] = 0.0;
    }
}

// alpha_j for columns still iterating; the test at the top of the oracle's
// loop (||r|| <= tol ||y||) and its pq <= 0 exit, per column.
__global__ void k_cg_alpha(int r, double tol, double *cg) {
    int j = threadIdx.x;
    if (j >= r) return;
    bool act = cg[CG_BROKEN * 32 + j] == 0.0 &&
               sqrt(cg[CG_RR * 32 + j]) > tol * sqrt(cg[CG_YY * 32 + j]);
    double pq = cg[CG_PQ * 32 + j];
    if (act && !(pq > 0.0)) {
        cg[CG_BROKEN * 32 + j] = 1.0;
        act = false;
    }
    cg[CG_ACT * 32 + j] = act ? 1.0 : 0.0;
    cg[CG_ALPHA * 32 + j] = act ? cg[CG_RZ * 32 + j] / pq : 0.0;
    if (act) cg[CG_IT * 32 + j] += 1.0;
}

__global__ void k_cg_beta(int r, double tol, double *cg) {
    int j = threadIdx.x;
    __shared__ int nact;
    if (j == 0) nact = 0;
    __syncthreads();
    if (j < r) {
        bool act = cg[CG_ACT * 32 + j] != 0.0;
        double rzn = cg[CG_RZN * 32 + j];
        cg[CG_ALPHA * 32 + j] = act ? rzn / cg[CG_RZ * 32 + j] : 0.0;   // beta, reuses the slot
        if (act) cg[CG_RZ * 32 + j] = rzn;
        bool next = cg[CG_BROKEN * 32 + j] == 0.0 &&
                    sqrt(cg[CG_RR * 32 + j]) > tol * sqrt(cg[CG_YY * 32 + j]);
        if (next) atomicAdd(&nact, 1);
    }
    __syncthreads();
    if (j == 0) cg[CG_NACT * 32] = (double)nact;
}

// X += alpha P, R -= alpha Q, Z = R   (per-column alpha)
template <typename T>
__global__ void k_cg_update(int64_t total, int r, const double *alpha, T *X, T *Rr, const T *P,
                            const T *Q, T *Z) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int j = (int)(i % r);
    T a = (T)alpha[j];
    T x = X[i], rr = Rr[i];
    if (a != (T)0) {
        x += a * P[i];
        rr -= a * Q[i];
        X[i] = x;
        Rr[i] = rr;
    }
    Z[i] = rr;
}

// P = Z + beta P for active columns
template <typename T>
__global__ void k_cg_p(int64_t total, int r, const double *beta, const double *act, const T *Z,
                       T *P) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int j = (int)(i % r);
    if (act[j] == 0.0) return;
    P[i] = Z[i] + (T)beta[j] * P[i];
}

template <typename T>
__global__ void k_zero(int64_t total, T *X) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) X[i] = (T)0;
}

static size_t esize(grass_prec p) { return p == GRASS_FP64 ? 8 : 4; }

int64_t s_solve(grass_ctx_t ctx, grass_sparsifier_t S, bool with_D, int r, grass_prec prec,
                const void *Y, void *X, double tol, int maxit, unsigned long long *maxbits) {
    grass_tree_t T = S->tree;
    const GraphData &g = T->g;
    const int64_t n = g.n, total = n * r;
    const size_t es = esize(prec);
    const TreeFactor &f = with_D ? T->sdd : T->lap;
    if (S->is_tree) {
        copy_d(ctx, X, Y, total * es);
        tree_solve_inplace(ctx, T, f, r, prec, X, maxbits);
        return 0;
    }
    double *cg = ctx->scal.p + DS_CG;
    char *R = ctx->scr<char>(SCR_CG_R, total * es);
    char *Z = ctx->scr<char>(SCR_CG_Z, total * es);
    char *P = ctx->scr<char>(SCR_CG_P, total * es);
    char *Q = ctx->scr<char>(SCR_CG_Q, total * es);
    const void *w = prec == GRASS_FP64 ? (const void *)S->s_w64.p : (const void *)S->s_w32.p;
    const void *D = with_D ? (prec == GRASS_FP64 ? (const void *)g.D64.p : (const void *)g.D32.p)
                           : nullptr;
    int64_t grid = cdiv(total, kBlock);
    if (prec == GRASS_FP64) launch(ctx, k_zero<double>, grid, kBlock, 0, total, (double *)X);
    else launch(ctx, k_zero<float>, grid, kBlock, 0, total, (float *)X);
    copy_d(ctx, R, Y, total * es);
    copy_d(ctx, Z, Y, total * es);
    tree_solve_inplace(ctx, T, f, r, prec, Z, nullptr);
    copy_d(ctx, P, Z, total * es);
    dot_cols(ctx, r, prec, n, R, Z, cg + CG_RZ * 32);
    dot_cols(ctx, r, prec, n, R, R, cg + CG_RR * 32);
    launch(ctx, k_cg_init_scalars, 1, 32, 0, r, cg);
    const int kCheck = 8;
    for (int k = 0; k < maxit; ++k) {
        if (k > 0 && k % kCheck == 0) {
            double nact = 0;
            d2h(ctx, &nact, cg + CG_NACT * 32, sizeof(double));
            if (nact == 0) break;
        }
        lap_mm(ctx, r, prec, n, S->s_nnz, S->s_ptr.p, S->s_col.p, w, D, P, Q, nullptr,
               GRASS_KF_SPMM_S);
        dot_cols(ctx, r, prec, n, P, Q, cg + CG_PQ * 32);
        launch(ctx, k_cg_alpha, 1, 32, 0, r, tol, cg);
        if (prec == GRASS_FP64)
            launch(ctx, k_cg_update<double>, grid, kBlock, 0, total, r,
                   (const double *)(cg + CG_ALPHA * 32), (double *)X, (double *)R,
                   (const double *)P, (const double *)Q, (double *)Z);
        else
            launch(ctx, k_cg_update<float>, grid, kBlock, 0, total, r,
                   (const double *)(cg + CG_ALPHA * 32), (float *)X, (float *)R,
                   (const float *)P, (const float *)Q, (float *)Z);
        dot_cols(ctx, r, prec, n, R, R, cg + CG_RR * 32);
        tree_solve_inplace(ctx, T, f, r, prec, Z, nullptr);
        dot_cols(ctx, r, prec, n, R, Z, cg + CG_RZN * 32);
        launch(ctx, k_cg_beta, 1, 32, 0, r, tol, cg);
        if (prec == GRASS_FP64)
            launch(ctx, k_cg_p<double>, grid, kBlock, 0, total, r,
                   (const double *)(cg + CG_ALPHA * 32), (const double *)(cg + CG_ACT * 32),
                   (const double *)Z, (double *)P);
        else
            launch(ctx, k_cg_p<float>, grid, kBlock, 0, total, r,
                   (const double *)(cg + CG_ALPHA * 32), (const double *)(cg + CG_ACT * 32),
                   (const float *)Z, (float *)P);
    }
    if (maxbits) max_abs_bits(ctx, prec, total, X, maxbits);
    double its[32];
    d2h(ctx, its, cg + CG_IT * 32, r * sizeof(double));
    int64_t mx = 0;
    for (int j = 0; j < r; ++j) mx = std::max<int64_t>(mx, (int64_t)its[j]);
    return mx;
}

// ---------------------------------------------------------------- PCG

enum { P_PQ = 0, P_RR = 2, P_RZ0 = 4, P_RZ1 = 5, P_RZO = 6, P_BB = 8, P_EE = 10 };

// x += a p, r -= a q with a = num / den (device scalars)
template <typename T>
__global__ void k_pcg_axpy(int64_t n, const double *num, const double *den, T *x, T *rr,
                           const T *p, const T *q) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T a = (T)(*num / *den);
    x[i] += a * p[i];
    rr[i] -= a * q[i];
}

// p = z + beta p, beta = (rz_new - rzo) / rz_old  (rzo = 0 for the standard update)
template <typename T>
__global__ void k_pcg_p(int64_t n, const double *rzn, const double *rzo, const double *rzold,
                        const T *z, T *p) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double b = (*rzn - (rzo ? *rzo : 0.0)) / *rzold;
    p[i] = z[i] + (T)b * p[i];
}

__global__ void k_residual64(int64_t n, const double *b, const double *Ax, double *r) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = b[i] - Ax[i];
}

__global__ void k_add_f32(int64_t n, const float *e, double *x) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += (double)e[i];
}

// One PCG run on A (prec) for A e = rhs, e0 = 0, until ||r|| <= tol_abs or
// maxit.  Returns iterations; inner iterations accumulate into *inner.
template <typename T>
static int pcg_core(grass_ctx_t ctx, grass_sparsifier_t S, grass_prec prec, const T *rhs, T *e,
                    double tol_abs, int maxit, double inner_tol, int inner_maxit, int64_t *inner) {
    grass_tree_t Tr = S->tree;
    const GraphData &g = Tr->g;
    const int64_t n = g.n;
    const bool flexible = !S->is_tree;
    double *sc = ctx->scal.p + DS_RED;
    T *r = ctx->scr<T>(SCR_PCG_R, n);
    T *z = ctx->scr<T>(SCR_PCG_Z, n);
    T *p = ctx->scr<T>(SCR_PCG_P, n);
    T *q = ctx->scr<T>(SCR_PCG_Q, n);
    T *zold = ctx->scr<T>(SCR_PCG_ZOLD, n);
    const void *wA = prec == GRASS_FP64 ? (const void *)g.adj_w64.p : (const void *)g.adj_w32.p;
    const void *DA = prec == GRASS_FP64 ? (const void *)g.D64.p : (const void *)g.D32.p;
    int64_t grid = cdiv(n, kBlock);
    launch(ctx, k_zero<T>, grid, kBlock, 0, n, e);
    copy_d(ctx, r, rhs, n * sizeof(T));
    *inner += s_solve(ctx, S, true, 1, prec, r, z, inner_tol, inner_maxit, nullptr);
    copy_d(ctx, p, z, n * sizeof(T));
    int cur = 0;   // rz[cur] holds r.z
    dot_cols(ctx, 1, prec, n, r, z, sc + P_RZ0);
    dot_cols(ctx, 1, prec, n, r, r, sc + P_RR);
    int k = 0;
    for (; k < maxit; ++k) {
        double rr = 0;
        d2h(ctx, &rr, sc + P_RR, sizeof(double));
        if (std::sqrt(rr) <= tol_abs) break;
        lap_mm(ctx, 1, prec, n, 2 * g.m, g.adj_ptr.p, g.adj_col.p, wA, DA, p, q, nullptr,
               GRASS_KF_SPMM_G);
        dot_cols(ctx, 1, prec, n, p, q, sc + P_PQ);
        launch(ctx, k_pcg_axpy<T>, grid, kBlock, 0, n, (const double *)(sc + P_RZ0 + cur),
               (const double *)(sc + P_PQ), e, r, (const T *)p, (const T *)q);
        dot_cols(ctx, 1, prec, n, r, r, sc + P_RR);
        if (flexible) copy_d(ctx, zold, z, n * sizeof(T));
        *inner += s_solve(ctx, S, true, 1, prec, r, z, inner_tol, inner_maxit, nullptr);
        int nxt = 1 - cur;
        dot_cols(ctx, 1, prec, n, r, z, sc + P_RZ0 + nxt);
        if (flexible) dot_cols(ctx, 1, prec, n, r, zold, sc + P_RZO);
        launch(ctx, k_pcg_p<T>, grid, kBlock, 0, n, (const double *)(sc + P_RZ0 + nxt),
               flexible ? (const double *)(sc + P_RZO) : (const double *)nullptr,
               (const double *)(sc + P_RZ0 + cur), (const T *)z, p);
        cur = nxt;
    }
    return k;
}

static double true_relres(grass_ctx_t ctx, const GraphData &g, const double *b, const double *x,
                          double bnorm, double *rvec) {
    const int64_t n = g.n;
    double *Ax = ctx->scr<double>(SCR_PCG_E, n);
    lap_mm(ctx, 1, GRASS_FP64, n, 2 * g.m, g.adj_ptr.p, g.adj_col.p, g.adj_w64.p, g.D64.p, x, Ax,
           nullptr, GRASS_KF_SPMM_G);
    launch(ctx, k_residual64, cdiv(n, kBlock), kBlock, 0, n, b, (const double *)Ax, rvec);
    double *sc = ctx->scal.p + DS_RED;
    dot_cols(ctx, 1, GRASS_FP64, n, rvec, rvec, sc + P_EE);
    double rr = 0;
    d2h(ctx, &rr, sc + P_EE, sizeof(double));
    return std::sqrt(rr) / bnorm;
}

void pcg_solve(grass_ctx_t ctx, grass_sparsifier_t S, const double *b, double *x, double tol,
               int maxit, grass_prec prec, double refine_tol, double inner_tol, int inner_maxit,
               grass_solve_stats_t *st) {
    const GraphData &g = S->tree->g;
    const int64_t n = g.n;
    double *sc = ctx->scal.p + DS_RED;
    dot_cols(ctx, 1, GRASS_FP64, n, b, b, sc + P_BB);
    double bb = 0;
    d2h(ctx, &bb, sc + P_BB, sizeof(double));
    double bnorm = std::sqrt(bb);
    int64_t inner = 0;
    int iters = 0, passes = 0;
    double rel = 0.0;
    if (bnorm == 0.0) {
        memset_d(ctx, x, 0, n * sizeof(double));
    } else if (prec == GRASS_FP64) {
        iters = pcg_core<double>(ctx, S, prec, b, x, tol * bnorm, maxit, inner_tol, inner_maxit,
                                 &inner);
        double *rv = ctx->scr<double>(SCR_PCG_X, n);
        rel = true_relres(ctx, g, b, x, bnorm, rv);
    } else {
        // FP64 iterative refinement around FP32 PCG
        double *r64 = ctx->scr<double>(SCR_PCG_X, n);
        float *r32 = ctx->scr<float>(SCR_H, n);
        float *e32 = ctx->scr<float>(SCR_Y, n);
        memset_d(ctx, x, 0, n * sizeof(double));
        rel = 1.0;
        copy_d(ctx, r64, b, n * sizeof(double));
        while (true) {
            if (rel <= tol || iters >= maxit || passes >= 64) break;
            double rnorm = rel * bnorm;
            convert_block(ctx, GRASS_FP32, n, r64, r32);
            int it = pcg_core<float>(ctx, S, GRASS_FP32, r32, e32, refine_tol * rnorm,
                                     maxit - iters, inner_tol, inner_maxit, &inner);
            iters += it;
            ++passes;
            launch(ctx, k_add_f32, cdiv(n, kBlock), kBlock, 0, n, (const float *)e32, x);
            double prev = rel;
            rel = true_relres(ctx, g, b, x, bnorm, r64);
            if (it == 0 || !(rel < prev)) break;   // no progress possible in FP32
        }
    }
    if (st) {
        st->iters = iters;
        st->refinements = passes;
        st->inner_iters = inner;
        st->rel_resid_fp64 = rel;
    }
    if (!(rel <= tol)) fail(GRASS_ERR_NOT_CONVERGED, "PCG stopped at relative residual " + std::to_string(rel));
}

}  // namespace grass
