// amg_fused.cu -- PCG on A = L_G + D (Sec. V-A) preconditioned by one
// V-cycle of the sparsifier's aggregation multigrid (amg.cu; the paper's
// multigrid solver of the sparsifier, Sec. IV-C-1), the whole PCG pass in
// one cooperative launch: no host round trip and no launch per level.
//
// The iteration and the V-cycle are those of amg_pcg / vcycle_T (one
// weighted-Jacobi sweep before and one after each coarse correction); the
// sums over a row's entries, an aggregate's members or a row of the
// coarsest inverse run in index order in the thread form, and lane-strided
// with a fixed xor tree in the warp form, so results are deterministic but
// not bit-identical to the launch form.  The phases are merged:
//  * the pre-smoothing of level 0 from zero (x = omega D^-1 r) is written by
//    the phase that updates r;
//  * level l going down: residual phase (one row per item), then the
//    restriction phase, which also writes the next level's pre-smoothing
//    x = omega b / diag;
//  * level l going up: the prolongation x + x_c[agg] is formed on the fly
//    inside the post-smoothing sweep (at the row and at every neighbour,
//    whose coarse vertex comes with the column: aggcol[j] = agg[col[j]]);
//    level 0's sweep writes z and the partial sums of r.z;
//  * levels of at most amg_warp_n vertices take one warp per row (their
//    rows are long: they carry the fine edges between aggregates), the rest
//    one thread per row, two rows in flight (FP32; one for FP64);
//  * the coarsest dense solve takes one warp per row across the grid;
//    optionally the levels of at most amg_tail_n vertices run in block 0
//    with block barriers while the other blocks wait at the next grid
//    barrier.
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
    const int32_t *aggcol;         // [nnz] agg[col[j]]
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
    int64_t warp_n;                // levels of at most this many vertices: a warp per row
    double tol_abs;
    int maxit;
    double *part;                  // [2][gridDim.x][32]
    double *out;                   // [0] += iterations, [1] = final r.r
    unsigned int *bar;
    long long budget;
    int *err;
};

// Rows v0 + u st (u < U) of a CSR: s[u] = sum_j w_j x'_j over each row in j
// order, x'_j = x[col_j] (+ xc[agg[col_j]] with PRO).  Four entries of every
// row are loaded (indices and weights, then the gathers) before any sum: the
// fused kernel runs few threads per SM, so each keeps U rows in flight.
template <typename T, int U, bool PRO>
__device__ __forceinline__ void rows_wx(const int32_t *ptr, const int32_t *col, const T *w,
                                        const T *x, const int32_t *aggcol, const T *xc, int64_t n,
                                        int64_t v0, int64_t st, T (&s)[U]) {
    int32_t jb[U], je[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t v = v0 + u * st;
        const bool ok = v < n;
        jb[u] = ok ? ptr[v] : 0;
        je[u] = ok ? ptr[v + 1] : 0;
        s[u] = (T)0;
    }
    bool more = true;
    while (more) {
        int32_t c[U][4];
        T wv[U][4], xv[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool ok = jb[u] + k < je[u];
                c[u][k] = ok ? col[jb[u] + k] : 0;
                wv[u][k] = ok ? w[jb[u] + k] : (T)0;
            }
        }
        if constexpr (PRO) {
            // the entries' coarse vertices come with the columns (aggcol), so
            // x and the coarse correction are gathered in the same round
            int32_t ag[U][4];
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int k = 0; k < 4; ++k) ag[u][k] = jb[u] + k < je[u] ? aggcol[jb[u] + k] : 0;
            }
            T cv[U][4];
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const bool ok = jb[u] + k < je[u];
                    xv[u][k] = ok ? x[c[u][k]] : (T)0;
                    cv[u][k] = ok ? xc[ag[u][k]] : (T)0;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (jb[u] + k < je[u]) xv[u][k] = xv[u][k] + cv[u][k];
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int k = 0; k < 4; ++k) xv[u][k] = jb[u] + k < je[u] ? x[c[u][k]] : (T)0;
            }
        }
        more = false;
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (jb[u] + k < je[u]) s[u] += wv[u][k] * xv[u][k];
            jb[u] += 4;
            more = more || jb[u] < je[u];
        }
    }
}

// Rows v0 + u st of A's Laplacian part: s[u] = sum_j w_j (pv[u] - p[col_j])
// in j order (the fused PCG's SpMV form), loads of all U rows first.
template <typename T, int U>
__device__ __forceinline__ void rows_lap(const int32_t *ptr, const int32_t *col, const T *w,
                                         const T *p, int64_t n, int64_t v0, int64_t st,
                                         const T (&pv)[U], T (&s)[U]) {
    int32_t jb[U], je[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t v = v0 + u * st;
        const bool ok = v < n;
        jb[u] = ok ? ptr[v] : 0;
        je[u] = ok ? ptr[v + 1] : 0;
        s[u] = (T)0;
    }
    bool more = true;
    while (more) {
        int32_t c[U][4];
        T wv[U][4], xv[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool ok = jb[u] + k < je[u];
                c[u][k] = ok ? col[jb[u] + k] : 0;
                wv[u][k] = ok ? w[jb[u] + k] : (T)0;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int k = 0; k < 4; ++k) xv[u][k] = jb[u] + k < je[u] ? p[c[u][k]] : (T)0;
        }
        more = false;
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (jb[u] + k < je[u]) s[u] += wv[u][k] * (pv[u] - xv[u][k]);
            jb[u] += 4;
            more = more || jb[u] < je[u];
        }
    }
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

// Rows in flight per thread in the thread-form phases: two for FP32, one
// for FP64 (whose doubled registers made two slower: 116.8 against 109.7 ms
// for the 100^3 step's FP64 solve; FP32 63.9 against 65.8 ms with one)
template <typename T>
constexpr int kRowsInFlight = sizeof(T) == 4 ? 2 : 1;

// res = b - (diag x - sum w x_j) on level L
template <typename T>
__device__ __forceinline__ void ph_residual(const FLevel<T> &L, T *res, int64_t i0, int64_t st) {
    constexpr int U = kRowsInFlight<T>;
    for (int64_t v0 = i0; v0 < L.n; v0 += U * st) {
        T xo[U], bo[U], d[U], sm[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t v = v0 + u * st;
            const bool ok = v < L.n;
            xo[u] = ok ? L.x[v] : (T)0;
            bo[u] = ok ? L.b[v] : (T)0;
            d[u] = ok ? L.diag[v] : (T)0;
        }
        rows_wx<T, U, false>(L.ptr, L.col, L.w, L.x, nullptr, nullptr, L.n, v0, st, sm);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t v = v0 + u * st;
            if (v < L.n) res[v] = bo[u] - (d[u] * xo[u] - sm[u]);
        }
    }
}

// C.b[c] = sum of res over the members of c (member order); C.x[c] =
// omega C.b[c] / C.diag[c] unless C is the coarsest level.  Two coarse
// vertices per step, the first four members' loads of both first.
template <typename T>
__device__ __forceinline__ void ph_restrict(const FLevel<T> &L, const FLevel<T> &C, const T *res,
                                            bool coarsest, int64_t i0, int64_t st) {
    for (int64_t c0 = i0; c0 < C.n; c0 += 2 * st) {
        int32_t q0[2], q1[2], m[2][4];
        T v[2][4], dc[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t c = c0 + u * st;
            const bool ok = c < C.n;
            q0[u] = ok ? L.mptr[c] : 0;
            q1[u] = ok ? L.mptr[c + 1] : 0;
            dc[u] = ok && !coarsest ? C.diag[c] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
#pragma unroll
            for (int k = 0; k < 4; ++k) m[u][k] = q0[u] + k < q1[u] ? L.mem[q0[u] + k] : 0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
#pragma unroll
            for (int k = 0; k < 4; ++k) v[u][k] = q0[u] + k < q1[u] ? res[m[u][k]] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t c = c0 + u * st;
            if (c >= C.n) break;
            T acc = v[u][0];
#pragma unroll
            for (int k = 1; k < 4; ++k)
                if (q0[u] + k < q1[u]) acc += v[u][k];
            for (int32_t q = q0[u] + 4; q < q1[u]; ++q) acc += res[L.mem[q]];
            C.b[c] = acc;
            if (!coarsest) C.x[c] = jac0_of(acc, dc[u]);
        }
    }
}

// t = x' + omega (b - (diag x' - sum w x'_j)) / diag with x' = x + xc[agg];
// with rz, accumulates b t (level 0: r.z)
template <typename T>
__device__ __forceinline__ void ph_post(const FLevel<T> &L, const T *xc, int64_t i0, int64_t st,
                                        Acc<T> *rz) {
    constexpr int U = kRowsInFlight<T>;
    for (int64_t v0 = i0; v0 < L.n; v0 += U * st) {
        T xv[U], bv[U], d[U], sm[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t v = v0 + u * st;
            const bool ok = v < L.n;
            xv[u] = ok ? L.x[v] : (T)0;
            bv[u] = ok ? L.b[v] : (T)0;
            d[u] = ok ? L.diag[v] : (T)0;
            const int32_t ag = ok ? L.agg[v] : 0;
            if (ok) xv[u] = xv[u] + xc[ag];
        }
        rows_wx<T, U, true>(L.ptr, L.col, L.w, L.x, L.aggcol, xc, L.n, v0, st, sm);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t v = v0 + u * st;
            if (v >= L.n) break;
            const T o = d[u] > (T)0 ? xv[u] + (T)kOmegaF * (bv[u] - (d[u] * xv[u] - sm[u])) / d[u]
                                    : xv[u];
            L.t[v] = o;
            if (rz) rz->add_prod(bv[u], o);
        }
    }
}

// coarsest: t = Cinv b, one warp per row (lanes read the row coalesced and
// are summed by a fixed xor tree); warps w0, w0 + ws, ... of the caller
template <typename T>
__device__ __forceinline__ void ph_coarse(const FLevel<T> &L, const T *cinv, int64_t w0,
                                          int64_t ws, Acc<T> *rz) {
    const int64_t nc = L.n;
    const int lane = threadIdx.x & 31;
    for (int64_t i = w0; i < nc; i += ws) {
        T s = (T)0;
        for (int64_t j = lane; j < nc; j += 32) s += cinv[i * nc + j] * L.b[j];
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) {
            L.t[i] = s;
            if (rz) rz->add_prod(L.b[i], s);
        }
    }
}

// Warp forms of the three level phases for small levels, whose rows are
// long (their entries are the fine edges between aggregates): one warp per
// row (or per coarse vertex), lanes strided over the entries, the lane sums
// added by a fixed xor tree; warps w0, w0 + ws, ... of the caller.
template <typename T>
__device__ __forceinline__ T warp_sum(T s) {
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    return s;
}

template <typename T>
__device__ __forceinline__ void ph_residual_w(const FLevel<T> &L, T *res, int64_t w0, int64_t ws) {
    const int lane = threadIdx.x & 31;
    for (int64_t v = w0; v < L.n; v += ws) {
        const int32_t jb = L.ptr[v], je = L.ptr[v + 1];
        T s = (T)0;
        for (int32_t j = jb + lane; j < je; j += 32) s += L.w[j] * L.x[L.col[j]];
        s = warp_sum(s);
        if (lane == 0) res[v] = L.b[v] - (L.diag[v] * L.x[v] - s);
    }
}

template <typename T>
__device__ __forceinline__ void ph_restrict_w(const FLevel<T> &L, const FLevel<T> &C, const T *res,
                                              bool coarsest, int64_t w0, int64_t ws) {
    const int lane = threadIdx.x & 31;
    for (int64_t c = w0; c < C.n; c += ws) {
        const int32_t q0 = L.mptr[c], q1 = L.mptr[c + 1];
        T s = (T)0;
        for (int32_t q = q0 + lane; q < q1; q += 32) s += res[L.mem[q]];
        s = warp_sum(s);
        if (lane == 0) {
            C.b[c] = s;
            if (!coarsest) C.x[c] = jac0_of(s, C.diag[c]);
        }
    }
}

template <typename T>
__device__ __forceinline__ void ph_post_w(const FLevel<T> &L, const T *xc, int64_t w0, int64_t ws,
                                          Acc<T> *rz) {
    const int lane = threadIdx.x & 31;
    for (int64_t v = w0; v < L.n; v += ws) {
        const int32_t jb = L.ptr[v], je = L.ptr[v + 1];
        T s = (T)0;
        for (int32_t j = jb + lane; j < je; j += 32) s += L.w[j] * (L.x[L.col[j]] + xc[L.aggcol[j]]);
        s = warp_sum(s);
        if (lane == 0) {
            const T xv = L.x[v] + xc[L.agg[v]];
            const T d = L.diag[v], bv = L.b[v];
            const T o = d > (T)0 ? xv + (T)kOmegaF * (bv - (d * xv - s)) / d : xv;
            L.t[v] = o;
            if (rz) rz->add_prod(bv, o);
        }
    }
}

// One V-cycle on level 0's b (= r) into level 0's t (= z), level 0's x
// already pre-smoothed; rz gets this thread's part of r.z.  False: a grid
// barrier gave up (every block returns).
template <typename T>
__device__ bool vcycle_fused(const AmgPcgArgs<T> &a, const FLevels<T> &F, unsigned int &epoch,
                             Acc<T> &rz) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int L = a.L, lt = a.lt;
    const int64_t gw = gt >> 5, nw = nth >> 5;
    for (int l = 0; l < lt; ++l) {
        const bool last = l + 1 == L - 1;
        if (F.l[l].n <= a.warp_n) ph_residual_w(F.l[l], a.res, gw, nw);
        else ph_residual(F.l[l], a.res, gt, nth);
        if (!grid_sync(a.bar, a.budget, a.err, epoch)) return false;
        if (F.l[l + 1].n <= a.warp_n) ph_restrict_w(F.l[l], F.l[l + 1], a.res, last, gw, nw);
        else ph_restrict(F.l[l], F.l[l + 1], a.res, last, gt, nth);
        if (!grid_sync(a.bar, a.budget, a.err, epoch)) return false;
    }
    if (lt == L - 1) {
        // no level in the tail: the coarsest solve across the grid's warps
        ph_coarse(F.l[L - 1], a.cinv, gw, nw, L == 1 ? &rz : nullptr);
    } else if (blockIdx.x == 0) {
        const int64_t t0 = threadIdx.x, bs = blockDim.x;
        for (int l = lt; l < L - 1; ++l) {
            ph_residual(F.l[l], a.res, t0, bs);
            __syncthreads();
            ph_restrict(F.l[l], F.l[l + 1], a.res, l + 1 == L - 1, t0, bs);
            __syncthreads();
        }
        ph_coarse<T>(F.l[L - 1], a.cinv, t0 >> 5, bs >> 5, nullptr);
        __syncthreads();
        for (int l = L - 2; l >= lt; --l) {
            ph_post(F.l[l], F.l[l + 1].t, t0, bs, l == 0 ? &rz : nullptr);
            __syncthreads();
        }
    }
    if (!grid_sync(a.bar, a.budget, a.err, epoch)) return false;
    for (int l = lt - 1; l >= 0; --l) {
        if (F.l[l].n <= a.warp_n) ph_post_w(F.l[l], F.l[l + 1].t, gw, nw, l == 0 ? &rz : nullptr);
        else ph_post(F.l[l], F.l[l + 1].t, gt, nth, l == 0 ? &rz : nullptr);
        if (l > 0 && !grid_sync(a.bar, a.budget, a.err, epoch)) return false;
    }
    return true;
}

template <typename T>
__global__ void __launch_bounds__(kFusedMaxThreads, 1)
    k_amg_pcg_persist(AmgPcgArgs<T> a, FLevels<T> F) {
    __shared__ double s_red[32][32];
    __shared__ double s_v[4];
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
            if (!vcycle_fused(a, F, epoch, arz)) return;
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
            // q = A p, p.q (two rows per step, every load of both first)
            Acc<T> apq;
            for (int64_t v0 = gt; v0 < a.n; v0 += 2 * nth) {
                T pv[2], dv[2], sm[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int64_t v = v0 + u * nth;
                    const bool ok = v < a.n;
                    pv[u] = ok ? a.p[v] : (T)0;
                    dv[u] = ok ? a.aD[v] : (T)0;
                }
                rows_lap<T, 2>(a.aptr, a.acol, a.aw, a.p, a.n, v0, nth, pv, sm);
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int64_t v = v0 + u * nth;
                    if (v >= a.n) break;
                    const T qv = dv[u] * pv[u] + sm[u];
                    a.q[v] = qv;
                    apq.add_prod(pv[u], qv);
                }
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
            if (!vcycle_fused(a, F, epoch, arz)) return;
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
        f.aggcol = Lv.aggcol.p;
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
    a.warp_n = ctx->amg_warp_n;
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
    // roofline accounting, each array counted once per phase that touches it
    // (s bytes an element, n_l vertices and nnz_l entries on level l):
    //  residual: CSR + x, b, diag read, res written;
    //  restriction: member lists, res read, b (and x, diag) of level l+1;
    //  post-smoothing: CSR + the entries' coarse vertices (aggcol) + agg, x,
    //  b, diag read, x_c gathered, t written;
    //  coarsest: its dense inverse and two vectors;
    //  per outer iteration: SpMV with A (CSR + p, D read, q written), the
    //  update (e, r read and written, p, q, diag read, x written: 8 ns), the
    //  V-cycle and p = z + beta p (3 ns); the run starts with 7 ns and one
    //  V-cycle and its last iteration skips one V-cycle and p (about 4 ns
    //  net).
    {
        const double sz = (double)sizeof(T), ns = (double)n * sz;
        double vc = 0.0;
        for (int l = 0; l + 1 < L; ++l) {
            const double nl = (double)H.lv[l]->n, nn = (double)H.lv[l + 1]->n;
            const double csr = 4.0 * (nl + 1) + (double)H.lv[l]->nnz * (4.0 + sz);
            const bool coarsest = l + 2 == L;
            vc += csr + 4.0 * nl * sz;                                            // residual
            vc += 4.0 * (nn + 1) + 4.0 * nl + nl * sz + (coarsest ? 1.0 : 3.0) * nn * sz;
            const double nnz = (double)H.lv[l]->nnz;
            vc += csr + 4.0 * nnz + 4.0 * nl + 4.0 * nl * sz + nn * sz;           // post-smoothing
        }
        const double nc = (double)H.nc;
        vc += nc * nc * sz + 2.0 * nc * sz;
        const double spmv_a = 4.0 * (n + 1) + 2.0 * g.m * (4.0 + sz) + 3.0 * ns;
        const double per_outer = spmv_a + 8.0 * ns + vc + 3.0 * ns;
        if (ctx->tfam == GRASS_KF_PCG) {
            const size_t snap = ctx->iter_launches.size();
            ctx->t_snap(out, snap, 0);
            ctx->iter_launches.push_back({4.0 * ns, per_outer, snap});
        }
    }
    bool timed = ctx->t_begin(GRASS_KF_PCG, 0.0);
    void *args[] = {&a, &F};
    GCK(cudaLaunchCooperativeKernel((const void *)k_amg_pcg_persist<T>, dim3(grid), dim3(threads),
                                    args, 0, ctx->stream));
    ctx->launches++;
    ctx->t_end(timed);
    if (ctx->tfam == GRASS_KF_PCG) ctx->t_snap(out, ctx->iter_launches.back().slot, 1);
    double h[2] = {0.0, 0.0};
    d2h(ctx, h, out, sizeof(h));
    return (int)h[0];
}

template int amg_pcg_fused<double>(grass_ctx_t, grass_sparsifier_t, AmgHier &, const double *,
                                   double *, double, int);
template int amg_pcg_fused<float>(grass_ctx_t, grass_sparsifier_t, AmgHier &, const float *,
                                  float *, double, int);

}  // namespace grass
