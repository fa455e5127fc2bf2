// partition.cu -- spectral graph partitioning (Sec. V-F): an approximate
// Fiedler vector of A = L_G + D by a few inverse power iterations, each
// solve by the sparsifier-preconditioned PCG of krylov.cu, then the sign cut.
//
// For a graph Laplacian (D = 0) A is singular with null vector 1: every
// right-hand side is first made orthogonal to 1 (so the system is
// consistent), and PCG converges in the complement of 1 (its grounded
// preconditioner adds only constants, which A annihilates); the solution is
// projected again.  The vector is normalised after every step, with
// deterministic FP64 sums (fixed grid, fixed order).
#include <cmath>

#include "common.cuh"

namespace grass {

__global__ void k_fill_one(int64_t n, double *o) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = 1.0;
}

// y -= sum / n (sum: device scalar)
__global__ void k_center(int64_t n, double *y, const double *sum) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] -= *sum / (double)n;
}

// x = y / sqrt(sq) (sq: device scalar; a zero vector stays zero)
__global__ void k_unit(int64_t n, const double *y, const double *sq, double *x) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = *sq;
    x[i] = s > 0.0 ? y[i] / sqrt(s) : 0.0;
}

// side[i] = 1 where x[i] >= 0 (the sign cut), count += sides set
__global__ void k_sign_cut(int64_t n, const double *x, uint8_t *side, unsigned long long *count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool pos = i < n && x[i] >= 0.0;
    if (i < n) side[i] = pos ? 1 : 0;
    const unsigned int c = __popc(__ballot_sync(0xffffffffu, pos));
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

// x <- (x - mean x) / ||x - mean x|| in place, through y; returns nothing to
// the host (the sums stay on the device)
static void project_unit(grass_ctx_t ctx, int64_t n, double *y, double *x, const double *ones,
                         double *sc) {
    dot_cols(ctx, 1, GRASS_FP64, n, y, ones, sc);
    launch(ctx, k_center, cdiv(n, kBlock), kBlock, 0, n, y, (const double *)sc);
    dot_cols(ctx, 1, GRASS_FP64, n, y, y, sc + 1);
    launch(ctx, k_unit, cdiv(n, kBlock), kBlock, 0, n, (const double *)y, (const double *)(sc + 1), x);
}

}  // namespace grass

using namespace grass;

extern "C" grass_status grass_fiedler(grass_ctx_t ctx, grass_sparsifier_t S, const double *x0,
                                      int iters, double tol, int maxit, grass_prec prec,
                                      int inner_maxit, double *u_out, uint8_t *side_out,
                                      grass_fiedler_stats_t *stats) {
    if (!ctx || !S) return GRASS_ERR_INVALID;
    bool converged = true;
    std::string last;
    try {
        GCK(cudaSetDevice(ctx->device));
        if (S->tree->g.nseg != 1) fail(GRASS_ERR_INVALID, "a batch of graphs is not supported");
        if (!x0) fail(GRASS_ERR_INVALID, "null x0");
        if (iters < 1 || maxit < 1 || !(tol > 0.0)) fail(GRASS_ERR_INVALID, "iters, maxit >= 1, tol > 0");
        if (prec != GRASS_FP64 && prec != GRASS_FP32) fail(GRASS_ERR_INVALID, "bad prec");
        if (inner_maxit < 0) fail(GRASS_ERR_INVALID, "inner_maxit must be >= 0");
        const double t0 = now_ms();
        ensure_sdd(ctx, S->tree);
        const int64_t n = S->tree->g.n;
        double *x = ctx->scr<double>(SCR_PART_X, n);
        double *y = ctx->scr<double>(SCR_PART_Y, n);
        double *ones = ctx->scr<double>(SCR_PART_1, n);
        double *sc = ctx->scal.p + DS_RED + 48;   // [48, 49] sums of this call
        launch(ctx, k_fill_one, cdiv(n, kBlock), kBlock, 0, n, ones);
        copy_d(ctx, y, x0, n * sizeof(double));
        project_unit(ctx, n, y, x, ones, sc);
        grass_fiedler_stats_t st;
        std::memset(&st, 0, sizeof(st));
        for (int k = 0; k < iters; ++k) {
            grass_solve_stats_t ps;
            std::memset(&ps, 0, sizeof(ps));
            clear_timeout(ctx);
            try {
                pcg_solve(ctx, S, x, y, tol, maxit, prec, 1e-2, 1e-2, inner_maxit, &ps);
            } catch (const Error &e) {
                if (e.st != GRASS_ERR_NOT_CONVERGED) throw;
                converged = false;
                last = e.msg;
            }
            check_timeout(ctx);
            st.pcg_iters += ps.iters;
            st.iters_done = k + 1;
            st.worst_rel_resid = std::max(st.worst_rel_resid, ps.rel_resid_fp64);
            project_unit(ctx, n, y, x, ones, sc);
        }
        // Rayleigh quotient x^T L_G x (x has unit norm) and the sign cut
        double *q = ctx->scal.p + DS_RED + 16;
        quad_forms(ctx, GRASS_FP64, S, x, q);
        unsigned long long *cnt = reinterpret_cast<unsigned long long *>(ctx->scal.p + DS_RED + 50);
        memset_d(ctx, cnt, 0, sizeof(unsigned long long));
        uint8_t *side = side_out ? side_out : ctx->scr<uint8_t>(SCR_SIM_C, n + 1);
        launch(ctx, k_sign_cut, cdiv(n, kBlock), kBlock, 0, n, (const double *)x, side, cnt);
        if (u_out) copy_d(ctx, u_out, x, n * sizeof(double));
        double qq[2];
        unsigned long long pos = 0;
        d2h(ctx, qq, q, sizeof(qq));
        d2h(ctx, &pos, cnt, sizeof(pos));
        st.rayleigh = qq[0];
        st.n_pos = (int64_t)pos;
        st.n_neg = n - (int64_t)pos;
        st.ms = now_ms() - t0;
        if (stats) *stats = st;
        if (!converged) fail(GRASS_ERR_NOT_CONVERGED, last);
    } catch (const Error &e) {
        ctx->err = e.msg;
        return e.st;
    } catch (...) {
        ctx->err = "unexpected internal error";
        return GRASS_ERR_CUDA;
    }
    return GRASS_OK;
}
