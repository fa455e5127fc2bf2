// krylov.cu -- sparsifier solves (tree solve or tree-preconditioned CG over
// r columns) and the PCG solver of A = L_G + D (Sec. V-A).
#include <cmath>
#include <cstring>

#include "tree_solve.cuh"

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

// alpha_j for columns still iterating: the inner CG's stop test at the top
// of each iteration (a column stops once ||r|| <= tol ||y||, the inner
// solve's relative residual) and its exit on pq <= 0, per column.
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

// ---------------------------------------------------------------- fused CG
// The whole r-column CG on L_S (+D) with the tree preconditioner in one
// cooperative kernel: the same iteration as the multi-kernel version below,
// with every dot product reduced by every block from per-block partials in
// one fixed order (so all blocks hold identical scalars and agree on when to
// stop), and grid barriers between the phases.

template <typename T>
struct CGArgs {
    int64_t n;
    const int32_t *sptr, *scol;
    const T *sw, *D;
    const T *Y;
    T *X, *Rv, *Z, *P, *Q;
    double tol;
    int maxit;
    double *part;                // [2][gridDim.x][32]
    double *iter_acc;            // += max over columns of the iterations; iter_acc[1] += 1
                                 // when a column reached the iteration cap
    unsigned long long *maxbits; // optional max |X|
    EulerKArgs eu;               // scan-form tree solve (r = 1, no D)
    // one column, scan form: perm != nullptr when the solve runs in another
    // numbering (X, Rv, Z, P, Q and the CSR indexed by k, vertex perm[k]); Y
    // is then read and the result written to Xout in vertex ids
    const int32_t *perm;
    T *Xout;
};

// Per-block column sums of the thread partials v[e] (column c*EPT + e),
// written to out[0..R): lanes sharing c fold together (xor offsets >= TPR),
// then one thread per column adds the warps in order.
// TPR: lanes per group of columns (a thread of lane l holds columns
// (l mod TPR) * EPT ..), EPT = R / TPR.
template <int R, int TPR = Lay<R>::TPR>
__device__ __forceinline__ void block_cols(const double (&v)[R / TPR], int c,
                                           double (*s_red)[32], double *out) {
    constexpr int EPT = R / TPR;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        double x = v[e];
        for (int d = 16; d >= TPR; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
        if (lane < TPR) s_red[wid][lane * EPT + e] = x;
    }
    __syncthreads();
    if (threadIdx.x < R) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += s_red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

template <int R, int TPR = Lay<R>::TPR, typename T>
__device__ __forceinline__ void block_cols(const Acc<T> (&a)[R / TPR], int c,
                                           double (*s_red)[32], double *out) {
    double v[R / TPR];
#pragma unroll
    for (int e = 0; e < R / TPR; ++e) v[e] = a[e].value();
    block_cols<R, TPR>(v, c, s_red, out);
}

// Column sums over all blocks' partials (same order in every block): warp j
// takes column j, lanes stride over the blocks, fixed xor tree.
// The loads of up to U x 32 blocks are issued before the first add (one
// round trip per U x 32 blocks instead of one per 32); the order of the
// adds is the plain one (lane, lane + 32, ...).
template <int R>
__device__ inline void grid_cols(const double *part, double *s_out) {
    constexpr int U = R == 1 ? 8 : 2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid < R) {
        double s = 0.0;
        for (unsigned b0 = lane; b0 < gridDim.x; b0 += 32 * U) {
            double v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const unsigned b = b0 + 32 * u;
                v[u] = b < gridDim.x ? part[(int64_t)b * 32 + wid] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (b0 + 32 * u < gridDim.x) s += v[u];
        }
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) s_out[wid] = s;
    }
    __syncthreads();
}

// threads of k_cg_persist: the scan form and r > 1 columns keep 1024
template <int R, bool EU>
__host__ __device__ constexpr int cg_max_threads() { return (EU || R > 1) ? kPersistMaxThreads : kFusedMaxThreads; }

// Laplacian rows of a CSR (off-diagonal weights w, columns col) applied to
// x with stride S: q[u] += w_j (xi[u] - x[col_j * S]) over the entries
// [jb[u], je[u]) of each row, in j order.  The first K entries of every row
// (indices and weights, then the gathers) are loaded before any arithmetic;
// a longer row goes on K entries at a time.
template <typename T, int U, int K, int S>
__device__ __forceinline__ void lap_rows(const int32_t *col, const T *w, const T *x, int32_t (&jb)[U],
                                         const int32_t (&je)[U], const T (&xi)[U], T (&q)[U]) {
    bool more = true;
    while (more) {
        int32_t cc[U][K];
        T wv[U][K], xc[U][K];
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int32_t j = jb[u] + k;
                const bool v = j < je[u];
                cc[u][k] = v ? col[j] : 0;
                wv[u][k] = v ? w[j] : (T)0;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int k = 0; k < K; ++k) xc[u][k] = jb[u] + k < je[u] ? x[(int64_t)cc[u][k] * S] : (T)0;
        }
        more = false;
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (jb[u] + k < je[u]) q[u] += wv[u][k] * (xi[u] - xc[u][k]);
            jb[u] += K;
            more = more || jb[u] < je[u];
        }
    }
}

// Two column sums at once: warps 0..R-1 reduce part0 and warps R..2R-1
// part1 (each the same order as grid_cols), when the block has 2R warps.
template <int R>
__device__ inline void grid_cols2(const double *part0, double *s_out0, const double *part1,
                                  double *s_out1) {
    if (2 * R > (int)(blockDim.x >> 5)) {
        grid_cols<R>(part0, s_out0);
        grid_cols<R>(part1, s_out1);
        return;
    }
    constexpr int U = R == 1 ? 8 : 2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid < 2 * R) {
        const double *part = wid < R ? part0 : part1;
        const int col = wid < R ? wid : wid - R;
        double s = 0.0;
        for (unsigned b0 = lane; b0 < gridDim.x; b0 += 32 * U) {
            double v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const unsigned b = b0 + 32 * u;
                v[u] = b < gridDim.x ? part[(int64_t)b * 32 + col] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (b0 + 32 * u < gridDim.x) s += v[u];
        }
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) (wid < R ? s_out0 : s_out1)[col] = s;
    }
    __syncthreads();
}

// The whole inner CG as a device function of a cooperative grid (used by
// k_cg_persist and inside the fused PCG).  Returns false when a barrier wait
// ran out (the caller must return).  Ends without a trailing grid barrier:
// every element of X is last written (and read by the max |X| pass) by the
// thread that owns it under the element mapping (one column: the chunks of
// for_chunks; else rows slot, slot + nslots, ... and columns c*EPT ..), so
// a caller with the same mapping
// reads X at once.  preset: the caller has already set X = 0, R = Z = Y and
// passed a grid barrier since.
template <typename T, int R, bool EU = false>
__device__ __forceinline__ bool cg_dev(const CGArgs<T> &g, const TreeKArgs<T> &tk,
                                       unsigned int &epoch, T *ys, bool preset = false) {
    static_assert(!EU || R == 1, "the scan-form solve handles one column");
    constexpr int TPR = Lay<R>::TPR, EPT = Lay<R>::EPT;
    __shared__ double s_red[32][32];
    __shared__ double s_rz[32], s_rr[32], s_yy[32], s_pq[32], s_new[32], s_al[32];
    __shared__ int s_act[32], s_brk[32], s_it[32], s_nact;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = (int)(gt % TPR);
    const int64_t slot = gt / TPR, nslots = (int64_t)gridDim.x * blockDim.x / TPR;
    double *part0 = g.part, *part1 = g.part + (int64_t)gridDim.x * 32;
    double *mypart0 = part0 + (int64_t)blockIdx.x * 32, *mypart1 = part1 + (int64_t)blockIdx.x * 32;
    double mx = 0.0;
    // Element loops in chunks (for_chunks): one column (chunks of rows, the
    // mapping the fused PCG uses for the same vectors), or for FP32 and
    // r = 4, 8, 16, 32 the n x r array as flat 4-float chunks; the thread
    // count is a multiple of r / 4, so a thread's chunks all hold columns
    // c4 .. c4 + 3 (c4 = 4 (gt mod r/4)): NA sums per thread, laid out for
    // block_cols as groups of TPA lanes.
    constexpr bool CH1 = R == 1;
    constexpr bool CHR = sizeof(T) == 4 && (R == 4 || R == 8 || R == 16 || R == 32);
    constexpr bool CH = CH1 || CHR;
    constexpr int W = Chunk<T>::W;
    constexpr int NA = CHR ? 4 : EPT;
    constexpr int TPA = CHR ? R / 4 : TPR;
    const int64_t nel = CHR ? g.n * R : g.n;
    const int c4 = CHR ? (int)(gt % (R / 4)) * 4 : 0;
    Acc<T> acc0[NA], acc1[NA];

    if (!preset && CH) {
        for_chunks<T>(nel, gt, (int64_t)gridDim.x * blockDim.x, [&](int64_t i0, int cnt) {
            T y[W], zero[W] = {};
            bool gathered = false;
            if constexpr (EU) {
                if (g.perm) {
#pragma unroll
                    for (int w = 0; w < W; ++w) y[w] = w < cnt ? g.Y[g.perm[i0 + w]] : (T)0;
                    gathered = true;
                }
            }
            if (!gathered) ld_chunk(g.Y + i0, cnt, y);
            st_chunk(g.X + i0, cnt, zero);
            st_chunk(g.Rv + i0, cnt, y);
            st_chunk(g.Z + i0, cnt, y);
        });
        if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return false;
    } else if (!preset) {
        for (int64_t i = slot; i < g.n; i += nslots) {
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                int64_t k = i * R + c * EPT + e;
                T y = g.Y[k];
                g.X[k] = (T)0;
                g.Rv[k] = y;
                g.Z[k] = y;
            }
        }
        if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return false;
    }
    if (threadIdx.x < R) {
        s_brk[threadIdx.x] = 0;
        s_it[threadIdx.x] = 0;
    }
    // Iteration `it` starts with Z = M^{-1} R (the only call site of the
    // tree solve), then P (it = 0: P = Z; else P = Z + beta P), then the
    // stop test (a column goes on while ||r|| > tol ||y||), the product and the
    // updates.  After the updates the test is looked at once more, so no
    // solve is spent when no column goes on.
    for (int it = 0;; ++it) {
        // the scan form writes Z with the element loops' own mapping (no
        // barrier); the elimination rounds write out of order
        if constexpr (EU) {
            if (!euler_solve_dev<T, true>(g.eu, g.Z, tk.bar, tk.budget, tk.err, epoch, mx)) return false;
        } else {
            if (!tree_solve_dev<T, R, false>(tk, g.Z, epoch, mx, ys)) return false;
            if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return false;
        }
#pragma unroll
        for (int e = 0; e < NA; ++e) acc0[e] = acc1[e] = Acc<T>();
        if constexpr (CH) {
            for_chunks<T>(nel, gt, (int64_t)gridDim.x * blockDim.x, [&](int64_t i0, int cnt) {
                T z[W], rr[W];
                ld_chunk(g.Z + i0, cnt, z);
                ld_chunk(g.Rv + i0, cnt, rr);
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    if (w >= cnt) break;
                    acc0[CHR ? w : 0].add_prod(rr[w], z[w]);
                    if (it == 0) acc1[CHR ? w : 0].add_prod(rr[w], rr[w]);
                }
                if (it == 0) st_chunk(g.P + i0, cnt, z);
            });
        } else {
        for (int64_t i = slot; i < g.n; i += nslots) {
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                int64_t k = i * R + c * EPT + e;
                T z = g.Z[k], rr = g.Rv[k];
                acc0[e].add_prod(rr, z);
                if (it == 0) {
                    g.P[k] = z;
                    acc1[e].add_prod(rr, rr);
                }
            }
        }
        }
        block_cols<R, TPA>(acc0, c, s_red, mypart0);
        if (it == 0) block_cols<R, TPA>(acc1, c, s_red, mypart1);
        if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return false;
        if (it == 0) {
            grid_cols2<R>(part0, s_rz, part1, s_rr);
            if (threadIdx.x < R) s_yy[threadIdx.x] = s_rr[threadIdx.x];
            __syncthreads();
        } else {
            grid_cols<R>(part0, s_new);
            if (threadIdx.x < R) {
                int j = threadIdx.x;
                double beta = s_act[j] ? s_new[j] / s_rz[j] : 0.0;
                if (s_act[j]) s_rz[j] = s_new[j];
                s_al[j] = beta;
            }
            __syncthreads();
            if constexpr (CH1) {
                if (s_act[0]) {
                    const T be = (T)s_al[0];
                    for_chunks<T>(g.n, gt, (int64_t)gridDim.x * blockDim.x, [&](int64_t i0, int cnt) {
                        T z[W], pv[W];
                        ld_chunk(g.Z + i0, cnt, z);
                        ld_chunk(g.P + i0, cnt, pv);
#pragma unroll
                        for (int w = 0; w < W; ++w) pv[w] = z[w] + be * pv[w];
                        st_chunk(g.P + i0, cnt, pv);
                    });
                }
            } else if constexpr (CHR) {
                for_chunks<T>(nel, gt, (int64_t)gridDim.x * blockDim.x, [&](int64_t i0, int cnt) {
                    T z[W], pv[W];
                    ld_chunk(g.Z + i0, cnt, z);
                    ld_chunk(g.P + i0, cnt, pv);
#pragma unroll
                    for (int w = 0; w < W; ++w)
                        if (s_act[c4 + w]) pv[w] = z[w] + (T)s_al[c4 + w] * pv[w];
                    st_chunk(g.P + i0, cnt, pv);
                });
            } else {
            for (int64_t i = slot; i < g.n; i += nslots) {
#pragma unroll
                for (int e = 0; e < EPT; ++e) {
                    int j = c * EPT + e;
                    if (!s_act[j]) continue;
                    int64_t k = i * R + j;
                    g.P[k] = g.Z[k] + (T)s_al[j] * g.P[k];
                }
            }
            }
            if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return false;
        }
        if (it >= g.maxit) break;
        // stop test per column: a column goes on while ||r|| > tol ||y||
        if (threadIdx.x == 0) s_nact = 0;
        __syncthreads();
        if (threadIdx.x < R) {
            int j = threadIdx.x;
            int a = !s_brk[j] && sqrt(s_rr[j]) > g.tol * sqrt(s_yy[j]);
            s_act[j] = a;
            if (a) atomicAdd(&s_nact, 1);
        }
        __syncthreads();
        if (s_nact == 0) break;
        // Q = L_S P (+D), partial P.Q (row layout)
        Acc<T> accq[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) accq[e] = Acc<T>();
        if constexpr (EPT == 1 && (EU || cg_max_threads<R, EU>() <= kFusedMaxThreads)) {
            // two rows at a time, every load of both rows before the sums
            constexpr int K = 4;
            for (int64_t i0 = slot; i0 < g.n; i0 += 2 * nslots) {
                int32_t jb[2], je[2];
                T p0[2], q[2], dd[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int64_t i = i0 + u * nslots;
                    const bool ok = i < g.n;
                    p0[u] = ok ? g.P[i * R + c] : (T)0;
                    dd[u] = ok && g.D ? g.D[i] : (T)0;
                    jb[u] = ok ? g.sptr[i] : 0;
                    je[u] = ok ? g.sptr[i + 1] : 0;
                    q[u] = (T)0;
                }
                lap_rows<T, 2, K, R>(g.scol, g.sw, g.P + c, jb, je, p0, q);
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int64_t i = i0 + u * nslots;
                    if (i >= g.n) break;
                    if (g.D) q[u] += dd[u] * p0[u];
                    g.Q[i * R + c] = q[u];
                    accq[0].add_prod(p0[u], q[u]);
                }
            }
        } else {
        for (int64_t i = slot; i < g.n; i += nslots) {
            T p0[EPT], q[EPT];
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                p0[e] = g.P[i * R + c * EPT + e];
                q[e] = (T)0;
            }
            for (int32_t j = g.sptr[i]; j < g.sptr[i + 1]; ++j) {
                const T *pq = g.P + (int64_t)g.scol[j] * R + c * EPT;
                T w = g.sw[j];
#pragma unroll
                for (int e = 0; e < EPT; ++e) q[e] += w * (p0[e] - pq[e]);
            }
            if (g.D) {
                T dd = g.D[i];
#pragma unroll
                for (int e = 0; e < EPT; ++e) q[e] += dd * p0[e];
            }
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                g.Q[i * R + c * EPT + e] = q[e];
                accq[e].add_prod(p0[e], q[e]);
            }
        }
        }
        block_cols<R>(accq, c, s_red, mypart0);
        if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return false;
        grid_cols<R>(part0, s_pq);
        if (threadIdx.x < R) {
            int j = threadIdx.x;
            double pq = s_pq[j];
            if (s_act[j] && !(pq > 0.0)) {
                s_brk[j] = 1;
                s_act[j] = 0;
            }
            s_al[j] = s_act[j] ? s_rz[j] / pq : 0.0;
            if (s_act[j]) s_it[j] += 1;
        }
        __syncthreads();
        // X += alpha P, R -= alpha Q, Z = R, partial R.R
#pragma unroll
        for (int e = 0; e < NA; ++e) acc1[e] = Acc<T>();
        if constexpr (CHR) {
            for_chunks<T>(nel, gt, (int64_t)gridDim.x * blockDim.x, [&](int64_t i0, int cnt) {
                T rr[W], xv[W], pv[W], qv[W];
                ld_chunk(g.Rv + i0, cnt, rr);
                ld_chunk(g.X + i0, cnt, xv);
                ld_chunk(g.P + i0, cnt, pv);
                ld_chunk(g.Q + i0, cnt, qv);
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const T a = (T)s_al[c4 + w];
                    if (a != (T)0) {
                        xv[w] += a * pv[w];
                        rr[w] -= a * qv[w];
                    }
                }
                st_chunk(g.X + i0, cnt, xv);
                st_chunk(g.Rv + i0, cnt, rr);
                st_chunk(g.Z + i0, cnt, rr);
#pragma unroll
                for (int w = 0; w < W; ++w) acc1[w].add_prod(rr[w], rr[w]);
            });
        } else if constexpr (CH1) {
            const T a = (T)s_al[0];
            for_chunks<T>(g.n, gt, (int64_t)gridDim.x * blockDim.x, [&](int64_t i0, int cnt) {
                T rr[W];
                ld_chunk(g.Rv + i0, cnt, rr);
                if (a != (T)0) {
                    T xv[W], pv[W], qv[W];
                    ld_chunk(g.X + i0, cnt, xv);
                    ld_chunk(g.P + i0, cnt, pv);
                    ld_chunk(g.Q + i0, cnt, qv);
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        xv[w] += a * pv[w];
                        rr[w] -= a * qv[w];
                    }
                    st_chunk(g.X + i0, cnt, xv);
                    st_chunk(g.Rv + i0, cnt, rr);
                }
                st_chunk(g.Z + i0, cnt, rr);
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    if (w >= cnt) break;
                    acc1[0].add_prod(rr[w], rr[w]);
                }
            });
        } else {
        for (int64_t i = slot; i < g.n; i += nslots) {
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                int64_t k = i * R + c * EPT + e;
                T a = (T)s_al[c * EPT + e];
                T rr = g.Rv[k];
                if (a != (T)0) {
                    g.X[k] += a * g.P[k];
                    rr -= a * g.Q[k];
                    g.Rv[k] = rr;
                }
                g.Z[k] = rr;
                acc1[e].add_prod(rr, rr);
            }
        }
        }
        // look ahead: another iteration only if one is allowed and some
        // column passes the test
        if (it + 1 >= g.maxit) break;
        block_cols<R, TPA>(acc1, c, s_red, mypart1);
        if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return false;
        grid_cols<R>(part1, s_rr);
        if (threadIdx.x == 0) s_nact = 0;
        __syncthreads();
        if (threadIdx.x < R) {
            int j = threadIdx.x;
            if (!s_brk[j] && sqrt(s_rr[j]) > g.tol * sqrt(s_yy[j])) atomicAdd(&s_nact, 1);
        }
        __syncthreads();
        if (s_nact == 0) break;
    }
    if (g.maxbits) {
        double m = 0.0;
        if constexpr (CH) {
            for_chunks<T>(nel, gt, (int64_t)gridDim.x * blockDim.x, [&](int64_t i0, int cnt) {
                T xv[W];
                ld_chunk(g.X + i0, cnt, xv);
#pragma unroll
                for (int w = 0; w < W; ++w) m = fmax(m, fabs((double)xv[w]));
            });
        } else {
        for (int64_t i = slot; i < g.n; i += nslots) {
#pragma unroll
            for (int e = 0; e < EPT; ++e) m = fmax(m, fabs((double)g.X[i * R + c * EPT + e]));
        }
        }
        block_atomic_max(g.maxbits, m);
    }
    if constexpr (CH1 && EU) {
        // back to vertex ids: each thread scatters the elements it owns
        if (g.perm) {
            for_chunks<T>(g.n, gt, (int64_t)gridDim.x * blockDim.x, [&](int64_t i0, int cnt) {
                T xv[W];
                ld_chunk(g.X + i0, cnt, xv);
#pragma unroll
                for (int w = 0; w < W; ++w)
                    if (w < cnt) g.Xout[g.perm[i0 + w]] = xv[w];
            });
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int mxit = 0;
        for (int j = 0; j < R; ++j) mxit = max(mxit, s_it[j]);
        *g.iter_acc += (double)mxit;
        if (mxit >= g.maxit) g.iter_acc[1] += 1.0;
    }
    return true;
}

template <typename T, int R, bool EU>
__global__ void __launch_bounds__(cg_max_threads<R, EU>(), 1)
    k_cg_persist(CGArgs<T> g, TreeKArgs<T> tk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned int epoch = 0;
    if constexpr (!EU) tree_tail_stage<T, R>(tk, reinterpret_cast<T *>(smem_raw));
    cg_dev<T, R, EU>(g, tk, epoch, reinterpret_cast<T *>(smem_raw));
}

// S's adjacency in the tree's preorder numbering (row k = the row of vertex
// vert[k], columns renumbered, entries in their original order)
__global__ void k_pre_count(int64_t n, const int32_t *vert, const int32_t *sptr, int64_t *cnt) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) cnt[k] = sptr[vert[k] + 1] - sptr[vert[k]];
}

__global__ void k_pre_fill(int64_t n, const int32_t *vert, const int32_t *pre, const int32_t *sptr,
                           const int32_t *scol, const double *sw64, const float *sw32,
                           const int64_t *off, int32_t *pptr, int32_t *pcol, double *pw64,
                           float *pw32) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t v = vert[k];
    int64_t o = off[k];
    pptr[k] = (int32_t)o;
    if (k == n - 1) pptr[n] = (int32_t)off[n];
    for (int32_t j = sptr[v]; j < sptr[v + 1]; ++j, ++o) {
        pcol[o] = pre[scol[j]];
        pw64[o] = sw64[j];
        pw32[o] = sw32[j];
    }
}

static void sparsifier_pre(grass_ctx_t ctx, grass_sparsifier_t S) {
    if (S->pre_ok) return;
    const EulerTour &E = S->tree->euler;
    const int64_t n = S->tree->g.n;
    int64_t *cnt = ctx->scr<int64_t>(SCR_TMP2, n + 1);
    int64_t *off = ctx->scr<int64_t>(SCR_TMP3, n + 1);
    launch(ctx, k_pre_count, cdiv(n, kBlock), kBlock, 0, n, (const int32_t *)E.vert.p,
           (const int32_t *)S->s_ptr.p, cnt);
    int64_t nnz = 0;
    scan_i64(ctx, cnt, off, n, &nnz);
    if (nnz != S->s_nnz) fail(GRASS_ERR_CUDA, "preorder sparsifier: entry count mismatch");
    S->p_ptr.reserve(n + 1);
    S->p_col.reserve(nnz);
    S->p_w64.reserve(nnz);
    S->p_w32.reserve(nnz);
    launch(ctx, k_pre_fill, cdiv(n, kBlock), kBlock, 0, n, (const int32_t *)E.vert.p,
           (const int32_t *)E.pre.p, (const int32_t *)S->s_ptr.p, (const int32_t *)S->s_col.p,
           (const double *)S->s_w64.p, (const float *)S->s_w32.p, (const int64_t *)off,
           S->p_ptr.p, S->p_col.p, S->p_w64.p, S->p_w32.p);
    S->pre_ok = true;
}

template <typename T, int R>
static void cg_persistent(grass_ctx_t ctx, grass_sparsifier_t S, bool with_D, const void *Y,
                          void *X, double tol, int maxit, unsigned long long *maxbits) {
    grass_tree_t Tr = S->tree;
    const GraphData &g = Tr->g;
    const int64_t n = g.n;
    const TreeFactor &f = with_D ? Tr->sdd : Tr->lap;
    size_t smem = 0;
    TreeKArgs<T> tk = tree_kargs<T, R>(ctx, Tr, f, &smem);
    CGArgs<T> a;
    a.n = n;
    a.sptr = S->s_ptr.p;
    a.scol = S->s_col.p;
    const size_t total = (size_t)n * R;
    if constexpr (sizeof(T) == 8) {
        a.sw = S->s_w64.p;
        a.D = with_D ? g.D64.p : nullptr;
    } else {
        a.sw = S->s_w32.p;
        a.D = with_D ? g.D32.p : nullptr;
    }
    a.Y = (const T *)Y;
    a.X = (T *)X;
    a.Rv = ctx->scr<T>(SCR_CG_R, total);
    a.Z = ctx->scr<T>(SCR_CG_Z, total);
    a.P = ctx->scr<T>(SCR_CG_P, total);
    a.Q = ctx->scr<T>(SCR_CG_Q, total);
    a.tol = tol;
    a.maxit = maxit;
    a.part = ctx->partials.p;
    a.iter_acc = ctx->scal.p + DS_RED + DS_ITER;
    a.maxbits = maxbits;
    a.perm = nullptr;
    a.Xout = nullptr;
    std::memset(&a.eu, 0, sizeof(a.eu));
    // one column and no D: the scan-form tree solve, with the CG's vectors
    // and S in the tree's preorder (the tour then reads them in sequence);
    // Y is gathered at the start and X scattered at the end
    const bool eu = R == 1 && !with_D && ctx->euler_solve && Tr->euler.built;
    if (eu) {
        sparsifier_pre(ctx, S);
        a.sptr = S->p_ptr.p;
        a.scol = S->p_col.p;
        if constexpr (sizeof(T) == 8) a.sw = S->p_w64.p;
        else a.sw = S->p_w32.p;
        a.perm = Tr->euler.vert.p;
        a.Xout = (T *)X;
        a.X = ctx->scr<T>(SCR_CG_XP, total);
    }
    const int threads = bounded_threads(
        ctx->tree_threads, eu ? cg_max_threads<R, (R == 1)>() : cg_max_threads<R, false>());
    const void *kern = eu ? (const void *)k_cg_persist<T, R, (R == 1)>
                          : (const void *)k_cg_persist<T, R, false>;
    const int grid = eu ? coop_grid(ctx, k_cg_persist<T, R, (R == 1)>, threads, smem, n * Lay<R>::TPR)
                        : coop_grid(ctx, k_cg_persist<T, R, false>, threads, smem, n * Lay<R>::TPR);
    if ((size_t)grid * 32 * 2 > ctx->partials.n) fail(GRASS_ERR_CUDA, "partials buffer too small");
    // the chunked element loops (one FP32 column) take 16-byte accesses;
    // all their vectors are the context's own scratch (Y is gathered by
    // single loads when the solve runs in preorder)
    if (R == 1 && Chunk<T>::W > 1 &&
        (((a.perm ? (uintptr_t)0 : (uintptr_t)Y) | (uintptr_t)a.X | (uintptr_t)a.Rv |
          (uintptr_t)a.Z | (uintptr_t)a.P | (uintptr_t)a.Q) & 15))
        fail(GRASS_ERR_INVALID, "inner CG vectors must be 16-byte aligned");
    if (eu) euler_kargs<T>(ctx, Tr, grid, &a.eu, true);
    GCK(cudaMemsetAsync(tk.bar, 0, sizeof(unsigned int), ctx->stream));
    // roofline accounting, each array counted once per phase that touches
    // it: per iteration the tree solve, the SpMV with S (CSR, P read, Q
    // written, D), dots Z, R + P update Z, P, P + update R, X, P, Q read and
    // X, R, Z written (12 nrs; the first iteration's P = Z copies, 2 nrs
    // less); the start Y read and X, R, Z written (4 nrs); the end max |X|
    // (nrs) and, in preorder, the scatter of X (2 nrs)
    const TreeSchedule &TS = Tr->sched;
    const double s = (double)sizeof(T), nrs = (double)n * R * s;
    const double tree_b = 4.0 * nrs + TS.n_rcv * (16.0 + 2.0 * s) +
                          (n - (double)Tr->nroots) * (16.0 + 4.0 * s);
    const double spmv_b = 4.0 * (n + 1) + S->s_nnz * (4.0 + s) + 2.0 * nrs + (with_D ? n * s : 0.0);
    const bool timing = ctx->tfam == GRASS_KF_CG;
    size_t snap = ctx->iter_launches.size();
    if (timing) {
        ctx->t_snap(a.iter_acc, snap, 0);
        const double start = 2.0 * nrs + (maxbits ? nrs : 0.0) + (a.perm ? 2.0 * nrs : 0.0);
        ctx->iter_launches.push_back({start, tree_b + spmv_b + 12.0 * nrs, snap});
    }
    bool timed = ctx->t_begin(GRASS_KF_CG, 0.0);
    void *args[] = {&a, &tk};
    GCK(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(threads), args, smem, ctx->stream));
    ctx->launches++;
    ctx->t_end(timed);
    if (timing) ctx->t_snap(a.iter_acc, snap, 1);
}

struct CGCall {
    grass_ctx_t ctx;
    grass_sparsifier_t S;
    bool with_D;
    grass_prec prec;
    const void *Y;
    void *X;
    double tol;
    int maxit;
    unsigned long long *maxbits;
};

template <int R>
static void cg_R(const CGCall &c) {
    if (c.prec == GRASS_FP64)
        cg_persistent<double, R>(c.ctx, c.S, c.with_D, c.Y, c.X, c.tol, c.maxit, c.maxbits);
    else
        cg_persistent<float, R>(c.ctx, c.S, c.with_D, c.Y, c.X, c.tol, c.maxit, c.maxbits);
}

// acc[0] += the most iterations over the columns; acc[1] += 1 when a column
// reached the iteration cap (the capped-solve count of the fused kernels)
__global__ void k_acc_iters(int r, const double *cg_it, double maxit, double *acc) {
    double m = 0.0;
    for (int j = 0; j < r; ++j) m = fmax(m, cg_it[j]);
    acc[0] += m;
    if (m >= maxit) acc[1] += 1.0;
}

__global__ void k_f2d(int64_t n, const float *a, double *b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

__global__ void k_d2f(int64_t n, const double *a, float *b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// the inner-solve accumulators: iterations, and solves that reached the cap
__global__ void k_note_solve(double *acc, double its, double capped) {
    acc[0] += its;
    acc[1] += capped;
}

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
    if (ctx->lmax_amg && !with_D && r == 1) {
        // one column of L_S^+ by multigrid-preconditioned CG in FP64
        const double *y64 = (const double *)Y;
        double *x64 = (double *)X;
        if (prec == GRASS_FP32) {
            double *yb = ctx->scr<double>(SCR_AMG_Y, n);
            launch(ctx, k_f2d, cdiv(n, kBlock), kBlock, 0, n, (const float *)Y, yb);
            y64 = yb;
            x64 = ctx->scr<double>(SCR_AMG_X, n);
        }
        const int its = amg_cg_lap(ctx, S, y64, x64, tol, maxit);
        if (prec == GRASS_FP32) launch(ctx, k_d2f, cdiv(n, kBlock), kBlock, 0, n, (const double *)x64, (float *)X);
        if (maxbits) max_abs_bits(ctx, prec, n, X, maxbits);
        launch(ctx, k_note_solve, 1, 1, 0, ctx->scal.p + DS_RED + DS_ITER, (double)its,
               its >= maxit ? 1.0 : 0.0);
        return 0;
    }
    if (ctx->num_sms > 0) {
        CGCall call{ctx, S, with_D, prec, Y, X, tol, maxit, maxbits};
        GRASS_DISPATCH_R(r, cg_R, call);
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
               GRASS_KF_SPMM_S, &S->s_heavy);
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
    launch(ctx, k_acc_iters, 1, 1, 0, r, (const double *)(cg + CG_IT * 32), (double)maxit,
           ctx->scal.p + DS_RED + DS_ITER);
    return 0;
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

// ---------------------------------------------------------------- fused PCG
// The whole PCG run of pcg_core below in one cooperative launch: the same
// iteration (SpMV with A = L_G + D, alpha, updates, z = M^{-1} r by the
// tree solve or the inner CG device function, beta, p), every dot product
// reduced by every block from per-block partials in one fixed order, so all
// blocks hold the same scalars and stop together; no host round trip per
// iteration.

template <typename T>
struct PCGArgs {
    int64_t n;
    const int32_t *aptr, *acol;   // A = L_G + D: off-diagonal adjacency and D
    const T *aw, *aD;
    const T *rhs;
    T *e, *r, *z, *p, *q, *zo;
    double tol_abs;
    int maxit;
    double *part;                 // [2][gridDim.x][32]
    double *out;                  // [0] += iterations, [1] = final r.r
};

template <typename T, int MODE>
__global__ void __launch_bounds__(kFusedMaxThreads, 1)
    k_pcg_persist(PCGArgs<T> a, CGArgs<T> in, TreeKArgs<T> tk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *ys = reinterpret_cast<T *>(smem_raw);
    __shared__ double s_red[32][32];
    __shared__ double s_v[4];
    unsigned int epoch = 0;
    double mx = 0.0;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    double *P0 = a.part, *P1 = a.part + (int64_t)gridDim.x * 32;
    double *my0 = P0 + (int64_t)blockIdx.x * 32, *my1 = P1 + (int64_t)blockIdx.x * 32;
    Acc<T> acc0[1], acc1[1];
    constexpr int W = Chunk<T>::W;
    tree_tail_stage<T, 1>(tk, ys);

    // Element loops take the chunks of for_chunks (the inner CG's mapping).
    // e = 0, r = rhs; z = rhs for the tree solve, else the inner CG's start
    // (X = z = 0, R = Z = r)
    for_chunks<T>(a.n, gt, nth, [&](int64_t i0, int cnt) {
        T y[W], zero[W] = {};
        ld_chunk(a.rhs + i0, cnt, y);
        st_chunk(a.e + i0, cnt, zero);
        st_chunk(a.r + i0, cnt, y);
        if (MODE != 0) {
            st_chunk(a.z + i0, cnt, y);
        } else {
            st_chunk(a.z + i0, cnt, zero);
            st_chunk(in.Rv + i0, cnt, y);
            st_chunk(in.Z + i0, cnt, y);
        }
    });
    if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return;
    if constexpr (MODE == 2) {
        // One inner CG step from zero on (L_S + D), in closed form: with
        // z0 = T^{-1} r (the tree solve) the step is z = alpha_in z0,
        // alpha_in = r.z0 / z0'(L_S + D) z0.  One phase gives the quadratic
        // form (row by row) and r.z0, r.z0_prev (r.r on the first pass); the
        // outer scalars follow from them (r.z = alpha_in r.z0, r.z_old =
        // alpha_prev r.z0_prev).  z0 and z0_prev alternate between the two
        // buffers; the update writes the next solve's input r into the older.
        T *zc = a.z, *zp = a.zo;
        double rz = 0.0, rr = 0.0, aprev = 0.0;
        int k = 0, steps = 0;
        for (bool first = true;; first = false) {
            if (!tree_solve_dev<T, 1, false>(tk, zc, epoch, mx, ys)) return;
            if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return;
            Acc<T> aq, arz, ax;
            for (int64_t i0 = gt; i0 < a.n; i0 += 2 * nth) {
                constexpr int K = 4;
                int32_t jb[2], je[2];
                T zv[2], qv[2], dv[2], rv[2], ov[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int64_t i = i0 + u * nth;
                    const bool ok = i < a.n;
                    zv[u] = ok ? zc[i] : (T)0;
                    dv[u] = ok ? in.D[i] : (T)0;
                    rv[u] = ok ? a.r[i] : (T)0;
                    ov[u] = ok && !first ? zp[i] : (T)0;
                    jb[u] = ok ? in.sptr[i] : 0;
                    je[u] = ok ? in.sptr[i + 1] : 0;
                    qv[u] = (T)0;
                }
                lap_rows<T, 2, K, 1>(in.scol, in.sw, zc, jb, je, zv, qv);
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (i0 + u * nth >= a.n) break;
                    qv[u] += dv[u] * zv[u];
                    aq.add_prod(zv[u], qv[u]);
                    arz.add_prod(rv[u], zv[u]);
                    if (first) ax.add_prod(rv[u], rv[u]);
                    else ax.add_prod(rv[u], ov[u]);
                }
            }
            {
                double v4[4] = {aq.value(), arz.value(), ax.value(), 0.0};
                block_cols<4, 1>(v4, 0, s_red, my0);
            }
            if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return;
            __shared__ double s_q[4];
            grid_cols<4>(P0, s_q);
            const double quad = s_q[0], rz0 = s_q[1];
            const double ain = quad > 0.0 ? rz0 / quad : 0.0;
            const double rzn = ain * rz0;
            ++steps;
            T beta = (T)0;
            if (first) rr = s_q[2];
            else beta = (T)((rzn - aprev * s_q[2]) / rz);
            rz = rzn;
            aprev = ain;
            const T ai = (T)ain;
            // p = alpha_in z0 + beta p
            for_chunks<T>(a.n, gt, nth, [&](int64_t i0, int cnt) {
                T zv[W], pv[W];
                ld_chunk(zc + i0, cnt, zv);
                if (!first) ld_chunk(a.p + i0, cnt, pv);
#pragma unroll
                for (int w = 0; w < W; ++w) zv[w] = first ? ai * zv[w] : ai * zv[w] + beta * pv[w];
                st_chunk(a.p + i0, cnt, zv);
            });
            if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return;
            if (k >= a.maxit || sqrt(rr) <= a.tol_abs) break;
            // q = A p, pq (two rows at a time, every load of both rows first)
            acc0[0] = Acc<T>();
            for (int64_t i0 = gt; i0 < a.n; i0 += 2 * nth) {
                constexpr int K = 4;
                int32_t jb[2], je[2];
                T pv[2], qv[2], dv[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int64_t i = i0 + u * nth;
                    const bool ok = i < a.n;
                    pv[u] = ok ? a.p[i] : (T)0;
                    dv[u] = ok ? a.aD[i] : (T)0;
                    jb[u] = ok ? a.aptr[i] : 0;
                    je[u] = ok ? a.aptr[i + 1] : 0;
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) qv[u] = dv[u] * pv[u];
                lap_rows<T, 2, K, 1>(a.acol, a.aw, a.p, jb, je, pv, qv);
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int64_t i = i0 + u * nth;
                    if (i >= a.n) break;
                    a.q[i] = qv[u];
                    acc0[0].add_prod(pv[u], qv[u]);
                }
            }
            block_cols<1>(acc0, 0, s_red, my0);
            if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return;
            grid_cols<1>(P0, &s_v[2]);
            const T alpha = (T)(rz / s_v[2]);
            // e += alpha p, r -= alpha q, rr; the next solve's input r goes
            // into the buffer of z0_prev
            acc1[0] = Acc<T>();
            for_chunks<T>(a.n, gt, nth, [&](int64_t i0, int cnt) {
                T ev[W], pv[W], rv[W], qv[W];
                ld_chunk(a.e + i0, cnt, ev);
                ld_chunk(a.p + i0, cnt, pv);
                ld_chunk(a.r + i0, cnt, rv);
                ld_chunk(a.q + i0, cnt, qv);
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    ev[w] += alpha * pv[w];
                    rv[w] -= alpha * qv[w];
                }
                st_chunk(a.e + i0, cnt, ev);
                st_chunk(a.r + i0, cnt, rv);
                st_chunk(zp + i0, cnt, rv);
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    if (w >= cnt) break;
                    acc1[0].add_prod(rv[w], rv[w]);
                }
            });
            block_cols<1>(acc1, 0, s_red, my1);
            if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return;
            grid_cols<1>(P1, &s_v[3]);
            rr = s_v[3];
            T *t = zc;
            zc = zp;
            zp = t;
            ++k;
            if (k >= a.maxit || sqrt(rr) <= a.tol_abs) break;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.out[0] += (double)k;
            a.out[1] = rr;
            *in.iter_acc += (double)steps;
        }
        return;
    }
    // Each pass starts with z = M^{-1} r (the only call site of the
    // preconditioner), then p, then the test, the product and the updates;
    // the test is looked at once more after the updates, so no
    // preconditioner is applied once the run is over.
    double rz = 0.0, rr = 0.0;
    int k = 0;
    for (bool first = true;; first = false) {
        // the inner CG leaves every z[i] written by the thread that reads it
        // below; the tree solve writes out of order and needs the barrier
        if constexpr ((MODE == 1)) {
            if (!tree_solve_dev<T, 1, false>(tk, a.z, epoch, mx, ys)) return;
            if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return;
        } else {
            if (!cg_dev<T, 1>(in, tk, epoch, ys, true)) return;
        }
        // first: rz = r.z, rr = r.r;  later: r.z and r.z_old for beta
        acc0[0] = acc1[0] = Acc<T>();
        for_chunks<T>(a.n, gt, nth, [&](int64_t i0, int cnt) {
            T rv[W], zv[W], ov[W];
            ld_chunk(a.r + i0, cnt, rv);
            ld_chunk(a.z + i0, cnt, zv);
            if (!first && !(MODE == 1)) ld_chunk(a.zo + i0, cnt, ov);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                if (w >= cnt) break;
                acc0[0].add_prod(rv[w], zv[w]);
                if (first) acc1[0].add_prod(rv[w], rv[w]);
                else if (!(MODE == 1)) acc1[0].add_prod(rv[w], ov[w]);
            }
        });
        block_cols<1>(acc0, 0, s_red, my0);
        block_cols<1>(acc1, 0, s_red, my1);
        if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return;
        grid_cols2<1>(P0, &s_v[0], P1, &s_v[1]);
        const double rzn = s_v[0];
        T beta = (T)0;
        if (first) rr = s_v[1];
        else beta = (T)((rzn - ((MODE == 1) ? 0.0 : s_v[1])) / rz);
        rz = rzn;
        for_chunks<T>(a.n, gt, nth, [&](int64_t i0, int cnt) {
            T zv[W], pv[W];
            ld_chunk(a.z + i0, cnt, zv);
            if (!first) {
                ld_chunk(a.p + i0, cnt, pv);
#pragma unroll
                for (int w = 0; w < W; ++w) zv[w] += beta * pv[w];
            }
            st_chunk(a.p + i0, cnt, zv);
        });
        if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return;
        if (k >= a.maxit || sqrt(rr) <= a.tol_abs) break;
        // q = A p, pq
        // (two rows at a time, every load of both rows before the sums)
        acc0[0] = Acc<T>();
        for (int64_t i0 = gt; i0 < a.n; i0 += 2 * nth) {
            constexpr int K = 4;
            int32_t jb[2], je[2];
            T pv[2], qv[2], dv[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int64_t i = i0 + u * nth;
                const bool ok = i < a.n;
                pv[u] = ok ? a.p[i] : (T)0;
                dv[u] = ok ? a.aD[i] : (T)0;
                jb[u] = ok ? a.aptr[i] : 0;
                je[u] = ok ? a.aptr[i + 1] : 0;
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) qv[u] = dv[u] * pv[u];
            lap_rows<T, 2, K, 1>(a.acol, a.aw, a.p, jb, je, pv, qv);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int64_t i = i0 + u * nth;
                if (i >= a.n) break;
                a.q[i] = qv[u];
                acc0[0].add_prod(pv[u], qv[u]);
            }
        }
        block_cols<1>(acc0, 0, s_red, my0);
        if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return;
        grid_cols<1>(P0, &s_v[2]);
        const T alpha = (T)(rz / s_v[2]);
        // e += alpha p, r -= alpha q, rr; z = r for the tree solve, else
        // z_old = z and the next inner CG's start (X = z = 0, R = Z = r)
        acc1[0] = Acc<T>();
        for_chunks<T>(a.n, gt, nth, [&](int64_t i0, int cnt) {
            T ev[W], pv[W], rv[W], qv[W];
            ld_chunk(a.e + i0, cnt, ev);
            ld_chunk(a.p + i0, cnt, pv);
            ld_chunk(a.r + i0, cnt, rv);
            ld_chunk(a.q + i0, cnt, qv);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                ev[w] += alpha * pv[w];
                rv[w] -= alpha * qv[w];
            }
            st_chunk(a.e + i0, cnt, ev);
            st_chunk(a.r + i0, cnt, rv);
            if ((MODE == 1)) {
                st_chunk(a.z + i0, cnt, rv);
            } else {
                T zv[W], zero[W] = {};
                ld_chunk(a.z + i0, cnt, zv);
                st_chunk(a.zo + i0, cnt, zv);
                st_chunk(a.z + i0, cnt, zero);
                st_chunk(in.Rv + i0, cnt, rv);
                st_chunk(in.Z + i0, cnt, rv);
            }
#pragma unroll
            for (int w = 0; w < W; ++w) {
                if (w >= cnt) break;
                acc1[0].add_prod(rv[w], rv[w]);
            }
        });
        block_cols<1>(acc1, 0, s_red, my1);
        if (!grid_sync(tk.bar, tk.budget, tk.err, epoch)) return;
        grid_cols<1>(P1, &s_v[3]);
        rr = s_v[3];
        ++k;
        if (k >= a.maxit || sqrt(rr) <= a.tol_abs) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.out[0] += (double)k;
        a.out[1] = rr;
    }
}

// One PCG run on A (prec) for A e = rhs, e0 = 0, until ||r|| <= tol_abs or
// maxit.  Returns iterations; inner iterations accumulate into *inner.
template <typename T>
static int pcg_fused(grass_ctx_t ctx, grass_sparsifier_t S, const T *rhs, T *e, T *r, T *z, T *p,
                     T *q, T *zold, double tol_abs, int maxit, double inner_tol, int inner_maxit) {
    grass_tree_t Tr = S->tree;
    const GraphData &g = Tr->g;
    const int64_t n = g.n;
    size_t smem = 0;
    TreeKArgs<T> tk = tree_kargs<T, 1>(ctx, Tr, Tr->sdd, &smem);
    const int threads = bounded_threads(ctx->tree_threads, kFusedMaxThreads);
    // 1: the tree solve alone; 2: one inner CG step on the sparsifier, in
    // closed form; 0: the inner CG as a device function
    const int mode = (S->is_tree || inner_maxit <= 0) ? 1 : (inner_maxit == 1 ? 2 : 0);
    const void *kern = mode == 1 ? (const void *)k_pcg_persist<T, 1>
                     : mode == 2 ? (const void *)k_pcg_persist<T, 2>
                                 : (const void *)k_pcg_persist<T, 0>;
    const int grid = mode == 1 ? coop_grid(ctx, k_pcg_persist<T, 1>, threads, smem, n)
                   : mode == 2 ? coop_grid(ctx, k_pcg_persist<T, 2>, threads, smem, n)
                               : coop_grid(ctx, k_pcg_persist<T, 0>, threads, smem, n);
    PCGArgs<T> a;
    a.n = n;
    a.aptr = g.adj_ptr.p;
    a.acol = g.adj_col.p;
    CGArgs<T> in;
    std::memset(&in, 0, sizeof(in));
    in.n = n;
    if constexpr (sizeof(T) == 8) {
        a.aw = g.adj_w64.p;
        a.aD = g.D64.p;
        in.sw = S->s_w64.p;
        in.D = g.D64.p;
    } else {
        a.aw = g.adj_w32.p;
        a.aD = g.D32.p;
        in.sw = S->s_w32.p;
        in.D = g.D32.p;
    }
    a.rhs = rhs;
    a.e = e;
    a.r = r;
    a.z = z;
    a.p = p;
    a.q = q;
    a.zo = zold;
    a.tol_abs = tol_abs;
    a.maxit = maxit;
    a.part = ctx->scr<double>(SCR_PART2, (size_t)grid * 64);   // two [grid][32] partial arrays
    double *out = ctx->scal.p + DS_RED + DS_PCG;
    a.out = out;
    // the inner CG (sparsifier with off-tree edges): solves (L_S + D) z = r
    in.sptr = S->s_ptr.p;
    in.scol = S->s_col.p;
    in.Y = r;
    in.X = z;
    in.Rv = ctx->scr<T>(SCR_CG_R, n);
    in.Z = ctx->scr<T>(SCR_CG_Z, n);
    in.P = ctx->scr<T>(SCR_CG_P, n);
    in.Q = ctx->scr<T>(SCR_CG_Q, n);
    in.tol = inner_tol;
    in.maxit = inner_maxit;
    in.part = ctx->partials.p;
    in.iter_acc = ctx->scal.p + DS_RED + DS_ITER;
    in.maxbits = nullptr;
    if ((size_t)grid * 32 * 2 > ctx->partials.n) fail(GRASS_ERR_CUDA, "partials buffer too small");
    if (Chunk<T>::W > 1 && (((uintptr_t)rhs | (uintptr_t)e | (uintptr_t)r | (uintptr_t)z |
                             (uintptr_t)p | (uintptr_t)q | (uintptr_t)zold | (uintptr_t)in.Rv |
                             (uintptr_t)in.Z) & 15))
        fail(GRASS_ERR_INVALID, "PCG vectors must be 16-byte aligned");
    memset_d(ctx, out, 0, 2 * sizeof(double));
    GCK(cudaMemsetAsync(tk.bar, 0, sizeof(unsigned int), ctx->stream));
    // roofline accounting, each array counted once per phase that touches it
    // (s bytes an element): per outer iteration and per inner CG iteration.
    //  tree solve: tree_b;  SpMV with A: CSR + p, D read, q written;
    //  mode 1: dots r, z; p: z, p, p; update: e, p, r, q read, e, r, z
    //          written -> 12 ns;
    //  mode 2: the quadratic form over S's CSR with z, D read; dots r, z0_prev;
    //          p: z, p, p; update: e, p, r, q read, e, r, z written -> 14 ns;
    //  mode 0: outer dots r, z, z_old; p: z, p, p; update: e, p, r, q, z read,
    //          e, r, z_old, z, R, Z written -> 17 ns, less 2 ns for the inner
    //          CG's first iteration; inner: tree_b, SpMV with S, 12 ns.
    const TreeSchedule &TS = Tr->sched;
    const double s = (double)sizeof(T), ns = (double)n * s;
    const double tree_b = 4.0 * ns + TS.n_rcv * (16.0 + 2.0 * s) +
                          (n - (double)Tr->nroots) * (16.0 + 4.0 * s);
    const double spmv_a = 4.0 * (n + 1) + 2.0 * g.m * (4.0 + s) + 3.0 * ns;
    const double csr_s = 4.0 * (n + 1) + S->s_nnz * (4.0 + s);
    double per_outer, per_inner = 0.0, start;
    if (mode == 1) {
        per_outer = tree_b + spmv_a + 12.0 * ns;
        start = 4.0 * ns;
    } else if (mode == 2) {
        per_outer = tree_b + spmv_a + csr_s + 2.0 * ns + 12.0 * ns;
        start = 4.0 * ns;
    } else {
        per_outer = spmv_a + 15.0 * ns;
        per_inner = tree_b + csr_s + 3.0 * ns + 12.0 * ns;
        start = 6.0 * ns;
    }
    const bool timing = ctx->tfam == GRASS_KF_PCG;
    size_t snap = ctx->iter_launches.size();
    if (timing) {
        ctx->t_snap(out, snap, 0);
        ctx->t_snap(in.iter_acc, snap + 1, 0);
        ctx->iter_launches.push_back({start, per_outer, snap});
        ctx->iter_launches.push_back({0.0, per_inner, snap + 1});
    }
    bool timed = ctx->t_begin(GRASS_KF_PCG, 0.0);
    void *args[] = {&a, &in, &tk};
    GCK(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(threads), args, smem, ctx->stream));
    ctx->launches++;
    ctx->t_end(timed);
    if (timing) {
        ctx->t_snap(out, snap, 1);
        ctx->t_snap(in.iter_acc, snap + 1, 1);
    }
    double h[2] = {0.0, 0.0};
    d2h(ctx, h, out, sizeof(h));
    return (int)h[0];
}

template <typename T>
static int pcg_core(grass_ctx_t ctx, grass_sparsifier_t S, grass_prec prec, const T *rhs, T *e,
                    double tol_abs, int maxit, double inner_tol, int inner_maxit, int64_t *inner) {
    grass_tree_t Tr = S->tree;
    const GraphData &g = Tr->g;
    const int64_t n = g.n;
    // the sparsifier's multigrid V-cycle: a fixed SPD preconditioner (plain
    // PCG update); else the tree solve or the inner CG (flexible update)
    const bool amg = ctx->pcg_precond == 1 && !S->is_tree;
    const bool flexible = !amg && !S->is_tree && inner_maxit > 0;
    double *sc = ctx->scal.p + DS_RED;
    T *r = ctx->scr<T>(SCR_PCG_R, n);
    T *z = ctx->scr<T>(SCR_PCG_Z, n);
    T *p = ctx->scr<T>(SCR_PCG_P, n);
    T *q = ctx->scr<T>(SCR_PCG_Q, n);
    T *zold = ctx->scr<T>(SCR_PCG_ZOLD, n);
    if (amg) return amg_pcg<T>(ctx, S, rhs, e, tol_abs, maxit);
    if (ctx->num_sms > 0) return pcg_fused<T>(ctx, S, rhs, e, r, z, p, q, zold, tol_abs, maxit,
                                               inner_tol, inner_maxit);
    const void *wA = prec == GRASS_FP64 ? (const void *)g.adj_w64.p : (const void *)g.adj_w32.p;
    const void *DA = prec == GRASS_FP64 ? (const void *)g.D64.p : (const void *)g.D32.p;
    int64_t grid = cdiv(n, kBlock);
    // inner_maxit = 0: the tree solve alone
    auto precond = [&]() -> int64_t {
        if (amg) {
            amg_vcycle(ctx, S, true, prec, r, z);
            return 0;
        }
        if (inner_maxit > 0) return s_solve(ctx, S, true, 1, prec, r, z, inner_tol, inner_maxit, nullptr);
        copy_d(ctx, z, r, n * sizeof(T));
        tree_solve_inplace(ctx, Tr, Tr->sdd, 1, prec, z, nullptr);
        return 0;
    };
    launch(ctx, k_zero<T>, grid, kBlock, 0, n, e);
    copy_d(ctx, r, rhs, n * sizeof(T));
    *inner += precond();
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
               GRASS_KF_SPMM_G, &g.heavy);
        dot_cols(ctx, 1, prec, n, p, q, sc + P_PQ);
        launch(ctx, k_pcg_axpy<T>, grid, kBlock, 0, n, (const double *)(sc + P_RZ0 + cur),
               (const double *)(sc + P_PQ), e, r, (const T *)p, (const T *)q);
        dot_cols(ctx, 1, prec, n, r, r, sc + P_RR);
        if (flexible) copy_d(ctx, zold, z, n * sizeof(T));
        *inner += precond();
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
           nullptr, GRASS_KF_SPMM_G, &g.heavy);
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
    memset_d(ctx, ctx->scal.p + DS_RED + DS_ITER, 0, sizeof(double));
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
            // a singular A (graph Laplacian): keep the pass's right-hand side in
            // A's range, the complement of 1 (rounding puts a component along 1
            // into r, which no correction can cancel)
            if (g.lap_only) project_ones(ctx, n, r64);
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
        double acc = 0.0;
        d2h(ctx, &acc, ctx->scal.p + DS_RED + DS_ITER, sizeof(double));
        st->inner_iters = inner + (int64_t)acc;
        st->rel_resid_fp64 = rel;
    }
    if (!(rel <= tol)) fail(GRASS_ERR_NOT_CONVERGED, "PCG stopped at relative residual " + std::to_string(rel));
}

}  // namespace grass
