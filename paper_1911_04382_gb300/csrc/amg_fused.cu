// amg_fused.cu -- PCG on A = L_G + D (Sec. V-A) preconditioned by one
// V-cycle of the sparsifier's aggregation multigrid (amg.cu; the paper's
// multigrid solver of the sparsifier, Sec. IV-C-1), the whole PCG pass in
// one cooperative launch: no host round trip and no launch per level.
//
// The iteration and the V-cycle are those of amg_pcg / vcycle_T (one
// weighted-Jacobi sweep before and one after each coarse correction), with
// the same arithmetic per element in the same order; only the phases are
// merged:
//  * the pre-smoothing of level 0 from zero (x = omega D^-1 r) is written by
//    the phase that updates r;
//  * level l going down: residual phase (one row per item), then the
//    restriction phase, which also writes the next level's pre-smoothing
//    x = omega b / diag;
//  * level l going up: the prolongation x + x_c[agg] is formed on the fly
//    inside the post-smoothing sweep (at the row and at every neighbour);
//    level 0's sweep writes z and the partial sums of r.z;
//  * levels of at most tail_n vertices, the coarsest dense solve included,
//    run in block 0 with block barriers while the other blocks wait at the
//    next grid barrier.
// Dot products: thread accumulators (Acc), per-block partials, and every
// block sums all blocks' partials in one fixed order, so all blocks hold the
// same scalars and stop together.  Grid barriers are the bounded ones of
// common.cuh.
#include "common.cuh"
#include "tree_solve.cuh"

namespace grass {

constexpr double kOmegaF = 2.0 / 3.0;   // the smoother weight of amg.cu

template <typename T>
struct FLevel {
    int64_t n;
    const int32_t *ptr, *col;      // off-diagonal adjacency
    const T *w, *diag;             // weights; diagonal = weighted degree + D
    const int32_t *agg;            // [n] coarse vertex (not on the coarsest level)
    const int32_t *mptr, *mem;     // members of the next level's vertices
    T *b, *x, *t;                  // right-hand side, pre-smoothed iterate, result
};

template <typename T>
struct FLevels {
    FLevel<T> l[kAmgFusedLevels];
};

template <typename T>
struct AmgPcgArgs {
    int64_t n;
    const int32_t *aptr, *acol;    // A = L_G + D
    const T *aw, *aD;
    const T *rhs;
    T *e, *r, *z, *p, *q;
    T *res;                        // residual scratch, n entries (any level)
    const T *cinv;                 // coarsest level's dense (grounded) inverse
    int L;                         // levels (the last is the coarsest)
    int lt;                        // first level run by block 0 alone
    double tol_abs;
    int maxit;
    double *part;                  // [2][gridDim.x][32]
    double *out;                   // [0] += iterations, [1] = final r.r
    unsigned int *bar;
    long long budget;
    int *err;
};

// sum_j w_j x[col_j] over [jb, je), in j order; four entries' loads first
template <typename T>
__device__ __forceinline__ T row_wx(const int32_t *col, const T *w, const T *x, int32_t jb,
                                    int32_t je) {
    T s = (T)0;
    for (; jb < je; jb += 4) {
        int32_t c[4];
        T wv[4], xv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool ok = jb + k < je;
            c[k] = ok ? col[jb + k] : 0;
            wv[k] = ok ? w[jb + k] : (T)0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) xv[k] = jb + k < je ? x[c[k]] : (T)0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (jb + k < je) s += wv[k] * xv[k];
    }
    return s;
}

// the same sum over the prolonged iterate x_j + xc[agg_j]
template <typename T>
__device__ __forceinline__ T row_wx_pro(const int32_t *col, const T *w, const T *x,
                                        const int32_t *agg, const T *xc, int32_t jb, int32_t je) {
    T s = (T)0;
    for (; jb < je; jb += 4) {
        int32_t c[4], ag[4];
        T wv[4], xv[4], cv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool ok = jb + k < je;
            c[k] = ok ? col[jb + k] : 0;
            wv[k] = ok ? w[jb + k] : (T)0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool ok = jb + k < je;
            xv[k] = ok ? x[c[k]] : (T)0;
            ag[k] = ok ? agg[c[k]] : 0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) cv[k] = jb + k < je ? xc[ag[k]] : (T)0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (jb + k < je) s += wv[k] * (xv[k] + cv[k]);
    }
    return s;
}

template <typename T>
__device__ __forceinline__ T jac0_of(T b, T d) {
    return d > (T)0 ? (T)kOmegaF * b / d : (T)0;
}

// Per-block sums of up to 4 values into out[0..N), then (after a grid
// barrier) every block's sums of all blocks' partials, same order everywhere.
template <int N>
__device__ __forceinline__ void block_sums(const double (&v)[N], double (*s_red)[32], double *out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int e = 0; e < N; ++e) {
        double x = v[e];
        for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
        if (lane == 0) s_red[wid][e] = x;
    }
    __syncthreads();
    if (threadIdx.x < N) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += s_red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

template <int N>
__device__ __forceinline__ void grid_sums(const double *part, double *s_out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid < N) {
        double s = 0.0;
        for (unsigned b0 = lane; b0 < gridDim.x; b0 += 32 * 4) {
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned b = b0 + 32 * u;
                v[u] = b < gridDim.x ? part[(int64_t)b * 32 + wid] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (b0 + 32 * u < gridDim.x) s += v[u];
        }
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) s_out[wid] = s;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- V-cycle phases
// Each phase walks its items from item `i0` with stride `st` (the grid's
// threads, or block 0's).

// res = b - (diag x - sum w x_j) on level L
template <typename T>
__device__ __forceinline__ void ph_residual(const FLevel<T> &L, T *res, int64_t i0, int64_t st) {
    for (int64_t v = i0; v < L.n; v += st) {
        const T s = row_wx(L.col, L.w, L.x, L.ptr[v], L.ptr[v + 1]);
        res[v] = L.b[v] - (L.diag[v] * L.x[v] - s);
    }
}

// C.b[c] = sum of res over the members of c (member order); C.x[c] =
// omega C.b[c] / C.diag[c] unless C is the coarsest level
template <typename T>
__device__ __forceinline__ void ph_restrict(const FLevel<T> &L, const FLevel<T> &C, const T *res,
                                            bool coarsest, int64_t i0, int64_t st) {
    for (int64_t c = i0; c < C.n; c += st) {
        const int32_t q0 = L.mptr[c], q1 = L.mptr[c + 1];
        T v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = q0 + k < q1 ? res[L.mem[q0 + k]] : (T)0;
        T acc = v[0];
#pragma unroll
        for (int k = 1; k < 4; ++k)
            if (q0 + k < q1) acc += v[k];
        for (int32_t q = q0 + 4; q < q1; ++q) acc += res[L.mem[q]];
        C.b[c] = acc;
        if (!coarsest) C.x[c] = jac0_of(acc, C.diag[c]);
    }
}

// t = x' + omega (b - (diag x' - sum w x'_j)) / diag with x' = x + xc[agg];
// with rz, accumulates b t (level 0: r.z)
template <typename T>
__device__ __forceinline__ void ph_post(const FLevel<T> &L, const T *xc, int64_t i0, int64_t st,
                                        Acc<T> *rz) {
    for (int64_t v = i0; v < L.n; v += st) {
        const T s = row_wx_pro(L.col, L.w, L.x, L.agg, xc, L.ptr[v], L.ptr[v + 1]);
        const T xv = L.x[v] + xc[L.agg[v]];
        const T d = L.diag[v], bv = L.b[v];
        const T o = d > (T)0 ? xv + (T)kOmegaF * (bv - (d * xv - s)) / d : xv;
        L.t[v] = o;
        if (rz) rz->add_prod(bv, o);
    }
}

// coarsest: t = Cinv b (block 0; b staged in shared memory)
template <typename T>
__device__ __forceinline__ void ph_coarse(const FLevel<T> &L, const T *cinv, T *sb, Acc<T> *rz) {
    const int64_t nc = L.n;
    for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) sb[j] = L.b[j];
    __syncthreads();
    for (int64_t i = threadIdx.x; i < nc; i += blockDim.x) {
        T s = (T)0;
        for (int64_t j = 0; j < nc; ++j) s += cinv[i * nc + j] * sb[j];
        L.t[i] = s;
        if (rz) rz->add_prod(sb[i], s);
    }
}

// One V-cycle on level 0's b (= r) into level 0's t (= z), level 0's x
// already pre-smoothed; rz gets this thread's part of r.z.  False: a grid
// barrier gave up (every block returns).
template <typename T>
__device__ bool vcycle_fused(const AmgPcgArgs<T> &a, const FLevels<T> &F, unsigned int &epoch,
                             T *sb, Acc<T> &rz) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int L = a.L, lt = a.lt;
    for (int l = 0; l < lt; ++l) {
        ph_residual(F.l[l], a.res, gt, nth);
        if (!grid_sync(a.bar, a.budget, a.err, epoch)) return false;
        ph_restrict(F.l[l], F.l[l + 1], a.res, l + 1 == L - 1, gt, nth);
        if (!grid_sync(a.bar, a.budget, a.err, epoch)) return false;
    }
    if (blockIdx.x == 0) {
        const int64_t t0 = threadIdx.x, bs = blockDim.x;
        for (int l = lt; l < L - 1; ++l) {
            ph_residual(F.l[l], a.res, t0, bs);
            __syncthreads();
            ph_restrict(F.l[l], F.l[l + 1], a.res, l + 1 == L - 1, t0, bs);
            __syncthreads();
        }
        ph_coarse(F.l[L - 1], a.cinv, sb, L == 1 ? &rz : nullptr);
        __syncthreads();
        for (int l = L - 2; l >= lt; --l) {
            ph_post(F.l[l], F.l[l + 1].t, t0, bs, l == 0 ? &rz : nullptr);
            __syncthreads();
        }
    }
    if (!grid_sync(a.bar, a.budget, a.err, epoch)) return false;
    for (int l = lt - 1; l >= 0; --l) {
        ph_post(F.l[l], F.l[l + 1].t, gt, nth, l == 0 ? &rz : nullptr);
        if (l > 0 && !grid_sync(a.bar, a.budget, a.err, epoch)) return false;
    }
    return true;
}

template <typename T>
__global__ void __launch_bounds__(kFusedMaxThreads, 1)
    k_amg_pcg_persist(AmgPcgArgs<T> a, FLevels<T> F) {
    __shared__ double s_red[32][32];
    __shared__ double s_v[4];
    __shared__ T sb[kAmgCoarse];
    unsigned int epoch = 0;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    // two partial arrays: r.r of the update phase goes to the second, since
    // no grid barrier separates it from the reads of p.q in the first
    double *P0 = a.part, *P1 = a.part + (int64_t)gridDim.x * 32;
    double *my = P0 + (int64_t)blockIdx.x * 32, *my1 = P1 + (int64_t)blockIdx.x * 32;
    constexpr int W = Chunk<T>::W;
    const FLevel<T> &L0 = F.l[0];
    const double tol2 = a.tol_abs * a.tol_abs;

    // e = 0, r = rhs, level 0's pre-smoothing x = omega r / diag, r.r
    {
        Acc<T> arr;
        for_chunks<T>(a.n, gt, nth, [&](int64_t i0, int cnt) {
            T y[W], dv[W], xv[W], zero[W] = {};
            ld_chunk(a.rhs + i0, cnt, y);
            ld_chunk(L0.diag + i0, cnt, dv);
#pragma unroll
            for (int w = 0; w < W; ++w) xv[w] = jac0_of(y[w], dv[w]);
            st_chunk(a.e + i0, cnt, zero);
            st_chunk(a.r + i0, cnt, y);
            st_chunk(L0.x + i0, cnt, xv);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                if (w >= cnt) break;
                arr.add_prod(y[w], y[w]);
            }
        });
        double v1[1] = {arr.value()};
        block_sums<1>(v1, s_red, my);
    }
    if (!grid_sync(a.bar, a.budget, a.err, epoch)) return;
    grid_sums<1>(a.part, &s_v[0]);
    double rr = s_v[0];
    int k = 0;
    if (rr > tol2 && a.maxit > 0) {
        double rz = 0.0;
        {
            Acc<T> arz;
            if (!vcycle_fused(a, F, epoch, sb, arz)) return;
            double v1[1] = {arz.value()};
            block_sums<1>(v1, s_red, my);
            if (!grid_sync(a.bar, a.budget, a.err, epoch)) return;
            grid_sums<1>(a.part, &s_v[0]);
            rz = s_v[0];
        }
        // p = z
        for_chunks<T>(a.n, gt, nth, [&](int64_t i0, int cnt) {
            T zv[W];
            ld_chunk(a.z + i0, cnt, zv);
            st_chunk(a.p + i0, cnt, zv);
        });
        if (!grid_sync(a.bar, a.budget, a.err, epoch)) return;
        for (;;) {
            // q = A p, p.q
            Acc<T> apq;
            for (int64_t v = gt; v < a.n; v += nth) {
                const T pv = a.p[v];
                T qv = a.aD[v] * pv;
                const int32_t jb = a.aptr[v], je = a.aptr[v + 1];
                for (int32_t j0 = jb; j0 < je; j0 += 4) {
                    int32_t c[4];
                    T wv[4], xv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const bool ok = j0 + u < je;
                        c[u] = ok ? a.acol[j0 + u] : 0;
                        wv[u] = ok ? a.aw[j0 + u] : (T)0;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) xv[u] = j0 + u < je ? a.p[c[u]] : (T)0;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (j0 + u < je) qv += wv[u] * (pv - xv[u]);
                }
                a.q[v] = qv;
                apq.add_prod(pv, qv);
            }
            {
                double v1[1] = {apq.value()};
                block_sums<1>(v1, s_red, my);
            }
            if (!grid_sync(a.bar, a.budget, a.err, epoch)) return;
            grid_sums<1>(a.part, &s_v[1]);
            const T alpha = (T)(rz / s_v[1]);
            // e += alpha p, r -= alpha q, r.r, level 0's pre-smoothing
            Acc<T> arr;
            for_chunks<T>(a.n, gt, nth, [&](int64_t i0, int cnt) {
                T ev[W], pv[W], rv[W], qv[W], dv[W], xv[W];
                ld_chunk(a.e + i0, cnt, ev);
                ld_chunk(a.p + i0, cnt, pv);
                ld_chunk(a.r + i0, cnt, rv);
                ld_chunk(a.q + i0, cnt, qv);
                ld_chunk(L0.diag + i0, cnt, dv);
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    ev[w] += alpha * pv[w];
                    rv[w] -= alpha * qv[w];
                    xv[w] = jac0_of(rv[w], dv[w]);
                }
                st_chunk(a.e + i0, cnt, ev);
                st_chunk(a.r + i0, cnt, rv);
                st_chunk(L0.x + i0, cnt, xv);
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    if (w >= cnt) break;
                    arr.add_prod(rv[w], rv[w]);
                }
            });
            {
                double v1[1] = {arr.value()};
                block_sums<1>(v1, s_red, my1);
            }
            if (!grid_sync(a.bar, a.budget, a.err, epoch)) return;
            grid_sums<1>(P1, &s_v[2]);
            rr = s_v[2];
            ++k;
            if (!(rr > tol2) || k >= a.maxit) break;
            // z = V-cycle(r), r.z
            Acc<T> arz;
            if (!vcycle_fused(a, F, epoch, sb, arz)) return;
            {
                double v1[1] = {arz.value()};
                block_sums<1>(v1, s_red, my);
            }
            if (!grid_sync(a.bar, a.budget, a.err, epoch)) return;
            grid_sums<1>(a.part, &s_v[3]);
            const double rzn = s_v[3];
            const T beta = (T)(rzn / rz);
            rz = rzn;
            // p = z + beta p
            for_chunks<T>(a.n, gt, nth, [&](int64_t i0, int cnt) {
                T zv[W], pv[W];
                ld_chunk(a.z + i0, cnt, zv);
                ld_chunk(a.p + i0, cnt, pv);
#pragma unroll
                for (int w = 0; w < W; ++w) pv[w] = zv[w] + beta * pv[w];
                st_chunk(a.p + i0, cnt, pv);
            });
            if (!grid_sync(a.bar, a.budget, a.err, epoch)) return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.out[0] += (double)k;
        a.out[1] = rr;
    }
}

// ---------------------------------------------------------------- host

template <typename T>
int amg_pcg_fused(grass_ctx_t ctx, grass_sparsifier_t S, AmgHier &H, const T *rhs, T *e,
                  double tol_abs, int maxit) {
    const GraphData &g = S->tree->g;
    const int64_t n = g.n;
    const int L = (int)H.lv.size();
    if (L > kAmgFusedLevels) fail(GRASS_ERR_INVALID, "fused multigrid PCG: too many levels");
    AmgPcgArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    FLevels<T> F;
    std::memset(&F, 0, sizeof(F));
    a.n = n;
    a.aptr = g.adj_ptr.p;
    a.acol = g.adj_col.p;
    if constexpr (sizeof(T) == 8) {
        a.aw = g.adj_w64.p;
        a.aD = g.D64.p;
        a.cinv = H.cinv64.p;
    } else {
        a.aw = g.adj_w32.p;
        a.aD = g.D32.p;
        a.cinv = H.cinv32.p;
    }
    a.rhs = rhs;
    a.e = e;
    a.r = ctx->scr<T>(SCR_PCG_R, n);
    a.z = ctx->scr<T>(SCR_PCG_Z, n);
    a.p = ctx->scr<T>(SCR_PCG_P, n);
    a.q = ctx->scr<T>(SCR_PCG_Q, n);
    a.res = ctx->scr<T>(SCR_PCG_ZOLD, n);
    if (H.nc > kAmgCoarse) fail(GRASS_ERR_INVALID, "fused multigrid PCG: coarsest level too large");
    for (int l = 0; l < L; ++l) {
        AmgLevel &Lv = *H.lv[l];
        FLevel<T> &f = F.l[l];
        f.n = Lv.n;
        f.ptr = Lv.ptr.p;
        f.col = Lv.col.p;
        if constexpr (sizeof(T) == 8) {
            f.w = Lv.w64.p;
            f.diag = Lv.diag64.p;
        } else {
            f.w = Lv.w32.p;
            f.diag = Lv.diag32.p;
        }
        f.agg = Lv.agg.p;
        f.mptr = Lv.mptr.p;
        f.mem = Lv.mem.p;
        if (l == 0) {
            f.b = a.r;
            f.x = reinterpret_cast<T *>(Lv.vt.p);
            f.t = a.z;
        } else {
            f.b = reinterpret_cast<T *>(Lv.vb.p);
            f.x = reinterpret_cast<T *>(Lv.vx.p);
            f.t = reinterpret_cast<T *>(Lv.vt.p);
        }
    }
    // block 0 takes the levels from the first of at most amg_tail_n vertices
    a.L = L;
    a.lt = L - 1;
    for (int l = 0; l < L - 1; ++l)
        if (H.lv[l]->n <= ctx->amg_tail_n) {
            a.lt = l;
            break;
        }
    if (Chunk<T>::W > 1 && (((uintptr_t)rhs | (uintptr_t)e | (uintptr_t)a.r | (uintptr_t)a.z |
                             (uintptr_t)a.p | (uintptr_t)a.q | (uintptr_t)F.l[0].x |
                             (uintptr_t)F.l[0].diag) & 15))
        fail(GRASS_ERR_INVALID, "PCG vectors must be 16-byte aligned");
    const int threads = bounded_threads(ctx->tree_threads, kFusedMaxThreads);
    const int grid = coop_grid(ctx, k_amg_pcg_persist<T>, threads, 0, n);
    if ((size_t)grid * 64 > ctx->partials.n) fail(GRASS_ERR_CUDA, "partials buffer too small");
    a.part = ctx->partials.p;
    a.tol_abs = tol_abs;
    a.maxit = maxit;
    double *out = ctx->scal.p + DS_RED + DS_PCG;
    a.out = out;
    a.bar = ctx->gbar.p;
    a.budget = ctx->wait_budget;
    a.err = ctx->flags.p + 3;       // the timeout flag of the bounded waits
    memset_d(ctx, out, 0, 2 * sizeof(double));
    GCK(cudaMemsetAsync(a.bar, 0, sizeof(unsigned int), ctx->stream));
    bool timed = ctx->t_begin(GRASS_KF_PCG, 0.0);
    void *args[] = {&a, &F};
    GCK(cudaLaunchCooperativeKernel((const void *)k_amg_pcg_persist<T>, dim3(grid), dim3(threads),
                                    args, 0, ctx->stream));
    ctx->launches++;
    ctx->t_end(timed);
    double h[2] = {0.0, 0.0};
    d2h(ctx, h, out, sizeof(h));
    return (int)h[0];
}

template int amg_pcg_fused<double>(grass_ctx_t, grass_sparsifier_t, AmgHier &, const double *,
                                   double *, double, int);
template int amg_pcg_fused<float>(grass_ctx_t, grass_sparsifier_t, AmgHier &, const float *,
                                  float *, double, int);

}  // namespace grass
