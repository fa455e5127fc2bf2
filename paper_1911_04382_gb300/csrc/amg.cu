// amg.cu -- aggregation multigrid for the sparsifier's matrix M = L_S + D
// (or L_S alone), the sparsifier solver of Sec. IV-C-1 / IV-D step 1 (the
// paper factorises or multigrids the sparsifier), used as the PCG
// preconditioner of A = L_G + D (Sec. V-A) and for the lambda_max
// estimate's solves with L_S.
//
// Setup, level by level until at most kCoarse vertices remain:
//  1. heavy-edge matching: rounds in which every unmatched vertex names its
//     heaviest unmatched neighbour (weight descending, equal weights by a
//     fixed hash of the edge's end pair) and mutual choices are matched --
//     each matched edge is the heaviest at
//     both its ends among the remaining ones (a locally dominant matching;
//     the result does not depend on timing);
//  2. an unmatched vertex joins the pair of its heaviest matched neighbour
//     (its anchor; the same tie-break); a vertex with no matched neighbour
//     stays alone;
//  3. aggregates are numbered in order of their smallest vertex; members
//     are listed as: the pair's smaller id, the other, the joiners anchored
//     at the smaller in the order of its adjacency row, then those of the
//     other -- a fixed order, so every sum below is deterministic;
//  4. the coarse matrix P^T M P of the piecewise-constant P: coarse row c is
//     the members' rows in member order, entries to other aggregates only
//     (a pair joined by several fine edges keeps them as separate entries),
//     coarse D = the members' summed D, diagonal = coarse D + row weights.
// The coarsest matrix is inverted densely (Gauss-Jordan, one block); for a
// Laplacian (D = 0 on the whole level) its last vertex is grounded first,
// which changes the coarse solution by a constant only.
//
// V-cycle from zero: nu weighted-Jacobi sweeps (omega = 2/3; the first one is
// x = omega D^-1 b), residual restricted to the coarse level (one kernel over
// the members), recursion, prolongation x += x_c[agg], nu sweeps.  The cycle
// is symmetric, so it is a fixed SPD (on the complement of 1 for a
// Laplacian) preconditioner for CG.
#include <cmath>

#include "common.cuh"
#include "tree_solve.cuh"

namespace grass {

constexpr int64_t kCoarse = kAmgCoarse;   // the coarsest level has at most this many vertices
constexpr int kMaxLevels = 40;
constexpr int kMatchRounds = 8;
constexpr double kOmega = 2.0 / 3.0;

// ---------------------------------------------------------------- setup kernels

// Tie-break key of the edge {a, b}: the SplitMix64 output mix (Steele, Lea
// and Flood) of the ordered pair, the same from both ends.  Equal weights
// then rank the edges in a scattered but fixed order, so a round of
// locally dominant edges matches a share of every chain instead of only
// the pair at its smaller end (which a plain smaller-id rule gives on
// unit-weight meshes, stalling the coarsening).
__device__ __forceinline__ unsigned long long pair_key(int32_t a, int32_t b) {
    unsigned long long z = ((unsigned long long)(uint32_t)min(a, b) << 32) | (uint32_t)max(a, b);
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// heavier (w, then the larger pair key) than the current best?
__device__ __forceinline__ bool better(double w, unsigned long long k, double bw,
                                       unsigned long long bk) {
    return w > bw || (w == bw && k > bk);
}

__global__ void k_amg_diag(int64_t n, const int32_t *ptr, const double *w, const double *D,
                           double *diag) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    double s = D ? D[v] : 0.0;
    for (int32_t j = ptr[v]; j < ptr[v + 1]; ++j) s += w[j];
    diag[v] = s;
}

// go: the previous round matched something (rounds after one that matched
// nothing would match nothing either, so they return at once)
__global__ void k_amg_cand(int64_t n, const int32_t *ptr, const int32_t *col, const double *w,
                           const int32_t *mate, int32_t *cand, const int *go) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || !*go) return;
    if (mate[v] >= 0) {
        cand[v] = -1;
        return;
    }
    double bw = -1.0;
    int32_t bu = -1;
    unsigned long long bk = 0;
    for (int32_t j = ptr[v]; j < ptr[v + 1]; ++j) {
        const int32_t u = col[j];
        if (u == v || mate[u] >= 0) continue;
        const unsigned long long k = pair_key((int32_t)v, u);
        if (bu < 0 || better(w[j], k, bw, bk)) {
            bw = w[j];
            bu = u;
            bk = k;
        }
    }
    cand[v] = bu;
}

__global__ void k_amg_pair(int64_t n, const int32_t *cand, int32_t *mate, const int *go,
                           int *changed) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || !*go || mate[v] >= 0) return;
    const int32_t u = cand[v];
    if (u >= 0 && cand[u] == (int32_t)v) {
        mate[v] = u;
        *changed = 1;
    }
}

// Warp forms of k_amg_cand, k_amg_ccount and k_amg_cfill for small levels,
// whose rows are long (they carry the fine edges between aggregates): one
// warp per vertex, lanes strided over the row.  They give the same results
// as the thread forms: the candidate is the heaviest by (w, pair key), the
// first in row order among equal ones (each lane keeps its first best, the
// lanes' bests are compared with the row position as the last key), and the
// coarse rows are written and their weights summed in row order.  Used on
// levels of at most ctx->amg_warp_setup_n vertices.
__global__ void k_amg_cand_w(int64_t n, const int32_t *ptr, const int32_t *col, const double *w,
                             const int32_t *mate, int32_t *cand, const int *go) {
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= n || !*go) return;
    if (mate[v] >= 0) {
        if (lane == 0) cand[v] = -1;
        return;
    }
    double bw = -1.0;
    int32_t bu = -1, bj = INT_MAX;
    unsigned long long bk = 0;
    for (int32_t j = ptr[v] + lane; j < ptr[v + 1]; j += 32) {
        const int32_t u = col[j];
        if (u == v || mate[u] >= 0) continue;
        const unsigned long long k = pair_key((int32_t)v, u);
        if (bu < 0 || better(w[j], k, bw, bk)) {
            bw = w[j];
            bu = u;
            bk = k;
            bj = j;
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        const double ow = __shfl_xor_sync(0xffffffffu, bw, d);
        const int32_t ou = __shfl_xor_sync(0xffffffffu, bu, d);
        const int32_t oj = __shfl_xor_sync(0xffffffffu, bj, d);
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, d);
        const bool take = ou >= 0 && (bu < 0 || better(ow, ok, bw, bk) ||
                                      (ow == bw && ok == bk && oj < bj));
        if (take) {
            bw = ow;
            bu = ou;
            bk = ok;
            bj = oj;
        }
    }
    if (lane == 0) cand[v] = bu;
}

__global__ void k_amg_ccount_w(int64_t nc, const int32_t *mptr, const int32_t *mem,
                               const int32_t *ptr, const int32_t *col, const int32_t *agg,
                               int64_t *ccnt) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= nc) return;
    int64_t k = 0;
    for (int32_t q = mptr[c]; q < mptr[c + 1]; ++q) {
        const int32_t v = mem[q];
        for (int32_t j = ptr[v] + lane; j < ptr[v + 1]; j += 32) k += agg[col[j]] != (int32_t)c;
    }
    for (int d = 16; d > 0; d >>= 1) k += __shfl_xor_sync(0xffffffffu, k, d);
    if (lane == 0) ccnt[c] = k;
}

__global__ void k_amg_cfill_w(int64_t nc, const int32_t *mptr, const int32_t *mem,
                              const int32_t *ptr, const int32_t *col, const double *w,
                              const double *D, const int32_t *agg, const int64_t *coff,
                              int32_t *cptr, int32_t *ccol, double *cw, double *cD, double *cdiag) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= nc) return;
    int64_t k = coff[c];
    if (lane == 0) {
        cptr[c] = (int32_t)k;
        if (c == nc - 1) cptr[nc] = (int32_t)coff[nc];
    }
    double dsum = 0.0, wsum = 0.0;
    for (int32_t q = mptr[c]; q < mptr[c + 1]; ++q) {
        const int32_t v = mem[q];
        dsum += D[v];
        const int32_t jb = ptr[v], je = ptr[v + 1];
        for (int32_t j0 = jb; j0 < je; j0 += 32) {
            const int32_t j = j0 + lane;
            int32_t a = 0;
            double wj = 0.0;
            bool keep = false;
            if (j < je) {
                a = agg[col[j]];
                wj = w[j];
                keep = a != (int32_t)c;
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int64_t at = k + __popc(m & ((1u << lane) - 1u));
                ccol[at] = a;
                cw[at] = wj;
            }
            // the kept weights added in row order
            for (int i = 0; i < 32; ++i) {
                const double wi = __shfl_sync(0xffffffffu, wj, i);
                if ((m >> i) & 1u) wsum += wi;
            }
            k += __popc(m);
        }
    }
    if (lane == 0) {
        cD[c] = dsum;
        cdiag[c] = dsum + wsum;
    }
}

// anchor[v]: for an unmatched v, its heaviest matched neighbour (-1: none);
// -2 for matched vertices.  leader[v]: smallest id of v's aggregate.
__global__ void k_amg_join(int64_t n, const int32_t *ptr, const int32_t *col, const double *w,
                           const int32_t *mate, int32_t *anchor, int32_t *leader) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    if (mate[v] >= 0) {
        anchor[v] = -2;
        leader[v] = min((int32_t)v, mate[v]);
        return;
    }
    double bw = -1.0;
    int32_t bu = -1;
    unsigned long long bk = 0;
    for (int32_t j = ptr[v]; j < ptr[v + 1]; ++j) {
        const int32_t u = col[j];
        if (u == v || mate[u] < 0) continue;
        const unsigned long long k = pair_key((int32_t)v, u);
        if (bu < 0 || better(w[j], k, bw, bk)) {
            bw = w[j];
            bu = u;
            bk = k;
        }
    }
    anchor[v] = bu;
    leader[v] = bu >= 0 ? min(bu, mate[bu]) : (int32_t)v;
}

// jslot[v]: rank of joiner v among the joiners anchored at its anchor, in the
// order of the anchor's row (first occurrence); jcount[u]: their number
__global__ void k_amg_slots(int64_t n, const int32_t *ptr, const int32_t *col, const int32_t *mate,
                            const int32_t *anchor, int32_t *jslot, int32_t *jcount) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int32_t c = 0;
    if (mate[u] >= 0) {
        for (int32_t j = ptr[u]; j < ptr[u + 1]; ++j) {
            const int32_t v = col[j];
            if (anchor[v] == (int32_t)u && jslot[v] < 0) jslot[v] = c++;
        }
    }
    jcount[u] = c;
}

__global__ void k_amg_leadflag(int64_t n, const int32_t *leader, int64_t *flag) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) flag[v] = leader[v] == (int32_t)v ? 1 : 0;
}

// agg[v] = number of the aggregate (pos of its leader); member counts
__global__ void k_amg_agg(int64_t n, const int32_t *leader, const int64_t *pos, const int32_t *mate,
                          const int32_t *jcount, int32_t *agg, int64_t *mcnt) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    agg[v] = (int32_t)pos[leader[v]];
    if (leader[v] == (int32_t)v) {
        const int32_t m = mate[v];
        mcnt[pos[v]] = 1 + (m >= 0 ? 1 + jcount[m] : 0) + jcount[v];
    }
}

__global__ void k_amg_members(int64_t n, const int32_t *leader, const int32_t *mate,
                              const int32_t *anchor, const int32_t *jslot, const int32_t *jcount,
                              const int32_t *agg, const int64_t *moff, int32_t *mem) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int64_t base = moff[agg[v]];
    const int32_t l = leader[v];
    const int32_t lm = mate[l];                       // the leader's mate (or -1)
    const int64_t pairs = lm >= 0 ? 2 : 1;
    if (anchor[v] == -2 || anchor[v] == -1) {         // matched, or alone
        mem[base + ((int32_t)v == l ? 0 : 1)] = (int32_t)v;
        return;
    }
    const int32_t a = anchor[v];
    mem[base + pairs + (a == l ? 0 : jcount[l]) + jslot[v]] = (int32_t)v;
}

// coarse row sizes: entries of the members' rows to other aggregates
__global__ void k_amg_ccount(int64_t nc, const int32_t *mptr, const int32_t *mem, const int32_t *ptr,
                             const int32_t *col, const int32_t *agg, int64_t *ccnt) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int64_t k = 0;
    for (int32_t q = mptr[c]; q < mptr[c + 1]; ++q) {
        const int32_t v = mem[q];
        for (int32_t j = ptr[v]; j < ptr[v + 1]; ++j) k += agg[col[j]] != (int32_t)c;
    }
    ccnt[c] = k;
}

__global__ void k_amg_cfill(int64_t nc, const int32_t *mptr, const int32_t *mem, const int32_t *ptr,
                            const int32_t *col, const double *w, const double *D,
                            const int32_t *agg, const int64_t *coff, int32_t *cptr, int32_t *ccol,
                            double *cw, double *cD, double *cdiag) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int64_t k = coff[c];
    cptr[c] = (int32_t)k;
    if (c == nc - 1) cptr[nc] = (int32_t)coff[nc];
    double dsum = 0.0, wsum = 0.0;
    for (int32_t q = mptr[c]; q < mptr[c + 1]; ++q) {
        const int32_t v = mem[q];
        dsum += D[v];
        for (int32_t j = ptr[v]; j < ptr[v + 1]; ++j) {
            const int32_t a = agg[col[j]];
            if (a == (int32_t)c) continue;
            ccol[k] = a;
            cw[k] = w[j];
            wsum += w[j];
            ++k;
        }
    }
    cD[c] = dsum;
    cdiag[c] = dsum + wsum;
}

__global__ void k_i64_to_i32(int64_t n, const int64_t *a, int32_t *b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (int32_t)a[i];
}

__global__ void k_amg_f32(int64_t n, const double *a, float *b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// dense coarsest matrix (row i by thread i, its entries added in row order;
// M zeroed before)
__global__ void k_amg_dense(int64_t nc, const int32_t *ptr, const int32_t *col, const double *w,
                            const double *diag, int ground, double *M) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    double *row = M + i * nc;
    if (ground && i == nc - 1) {
        row[i] = 1.0;
        return;
    }
    row[i] = diag[i];
    for (int32_t j = ptr[i]; j < ptr[i + 1]; ++j) {
        const int32_t c = col[j];
        if (ground && c == nc - 1) continue;
        row[c] -= w[j];
    }
}

// In-place Gauss-Jordan inverse of the SPD matrix M (nc x nc, one block; no
// pivoting: the pivots of an SPD matrix stay positive).  With `ground`, the
// grounded vertex's row and column of the inverse are then zeroed.
__global__ void k_amg_gauss_jordan(int64_t nc, double *M, int ground) {
    __shared__ double s_piv;
    for (int64_t p = 0; p < nc; ++p) {
        if (threadIdx.x == 0) s_piv = M[p * nc + p];
        __syncthreads();
        const double inv = 1.0 / s_piv;
        // row p: a_pj /= piv (j != p), a_pp = 1 / piv
        for (int64_t j = threadIdx.x; j < nc; j += blockDim.x)
            M[p * nc + j] = j == p ? inv : M[p * nc + j] * inv;
        __syncthreads();
        // other rows: a_ij -= a_ip a_pj (j != p); a_ip = -a_ip / piv
        for (int64_t e = threadIdx.x; e < nc * nc; e += blockDim.x) {
            const int64_t i = e / nc, j = e % nc;
            if (i == p || j == p) continue;
            M[e] -= M[i * nc + p] * M[p * nc + j];
        }
        __syncthreads();
        for (int64_t i = threadIdx.x; i < nc; i += blockDim.x)
            if (i != p) M[i * nc + p] = -M[i * nc + p] * inv;
        __syncthreads();
    }
    if (ground) {
        for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) {
            M[(nc - 1) * nc + j] = 0.0;
            M[j * nc + (nc - 1)] = 0.0;
        }
    }
}

// The same Gauss-Jordan inverse across a cooperative grid: step p reads the
// matrix after step p - 1 from one buffer and writes step p's into the other
// (one grid barrier a step, the same arithmetic per element as above); block
// b updates rows b, b + gridDim.x, ...  Returns through *which the buffer
// (0: M0, 1: M1) holding the inverse.  The FP64 work of the one-block form
// (about nc^3 multiply-adds) is spread over the SMs.
__global__ void k_amg_gj_grid(int64_t nc, double *M0, double *M1, unsigned int *bar, long long budget,
                              int *err) {
    __shared__ double rowp[kCoarse];
    unsigned int epoch = 0;
    for (int64_t p = 0; p < nc; ++p) {
        const double *src = (p & 1) ? M1 : M0;
        double *dst = (p & 1) ? M0 : M1;
        const double inv = 1.0 / src[p * nc + p];
        for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) rowp[j] = src[p * nc + j];
        __syncthreads();
        for (int64_t i = blockIdx.x; i < nc; i += gridDim.x) {
            const double aip = src[i * nc + p];
            for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) {
                double v;
                if (i == p) v = j == p ? inv : rowp[j] * inv;
                else if (j == p) v = -aip * inv;
                else v = src[i * nc + j] - aip * (rowp[j] * inv);
                dst[i * nc + j] = v;
            }
        }
        if (!grid_sync(bar, budget, err, epoch)) return;
    }
}

__global__ void k_amg_ground_inv(int64_t nc, double *M) {
    for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) {
        M[(nc - 1) * nc + j] = 0.0;
        M[j * nc + (nc - 1)] = 0.0;
    }
}

// ---------------------------------------------------------------- V-cycle kernels

template <typename T>
__global__ void k_jac0(int64_t n, const T *b, const T *diag, T *x) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) x[v] = diag[v] > (T)0 ? (T)kOmega * b[v] / diag[v] : (T)0;
}

// xo = x + omega (b - M x) / diag,  (M x)_v = diag_v x_v - sum_j w_vj x_j
template <typename T>
__global__ void k_jac(int64_t n, const int32_t *ptr, const int32_t *col, const T *w, const T *diag,
                      const T *b, const T *x, T *xo) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    T s = (T)0;
    for (int32_t j = ptr[v]; j < ptr[v + 1]; ++j) s += w[j] * x[col[j]];
    const T d = diag[v];
    xo[v] = d > (T)0 ? x[v] + (T)kOmega * (b[v] - (d * x[v] - s)) / d : x[v];
}

// res = b - M x, one row per thread
template <typename T>
__global__ void k_residual(int64_t n, const int32_t *ptr, const int32_t *col, const T *w,
                           const T *diag, const T *b, const T *x, T *res) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    T s = (T)0;
    for (int32_t j = ptr[v]; j < ptr[v + 1]; ++j) s += w[j] * x[col[j]];
    res[v] = b[v] - (diag[v] * x[v] - s);
}

// bc[c] = sum of res over the members of c, in member order (the first four
// gathers issued together)
template <typename T>
__global__ void k_restrict(int64_t nc, const int32_t *mptr, const int32_t *mem, const T *res,
                           T *bc) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int32_t q0 = mptr[c], q1 = mptr[c + 1];
    T v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = q0 + k < q1 ? res[mem[q0 + k]] : (T)0;
    T acc = v[0];
#pragma unroll
    for (int k = 1; k < 4; ++k)
        if (q0 + k < q1) acc += v[k];
    for (int32_t q = q0 + 4; q < q1; ++q) acc += res[mem[q]];
    bc[c] = acc;
}

template <typename T>
__global__ void k_prolong(int64_t n, const int32_t *agg, const T *xc, T *x) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) x[v] += xc[agg[v]];
}

// x = Cinv b for the coarsest level (one block; b staged in shared memory)
template <typename T>
__global__ void k_coarse_apply(int64_t nc, const T *Cinv, const T *b, T *x) {
    __shared__ T sb[kCoarse];
    for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) sb[j] = b[j];
    __syncthreads();
    for (int64_t i = threadIdx.x; i < nc; i += blockDim.x) {
        T s = (T)0;
        for (int64_t j = 0; j < nc; ++j) s += Cinv[i * nc + j] * sb[j];
        x[i] = s;
    }
}

// ---------------------------------------------------------------- setup

namespace {

template <typename T>
T *lvl_w(AmgLevel &L) {
    if constexpr (sizeof(T) == 8) return L.w64.p;
    else return L.w32.p;
}
template <typename T>
T *lvl_diag(AmgLevel &L) {
    if constexpr (sizeof(T) == 8) return L.diag64.p;
    else return L.diag32.p;
}

// level 0 from the sparsifier's adjacency (a copy: the hierarchy owns it)
std::unique_ptr<AmgLevel> level0(grass_ctx_t ctx, AmgHier &H, grass_sparsifier_t S, bool with_D) {
    const GraphData &g = S->tree->g;
    auto L = std::make_unique<AmgLevel>();
    L->n = g.n;
    L->nnz = S->s_nnz;
    H.arena.get(L->ptr, g.n + 1);
    H.arena.get(L->col, S->s_nnz);
    H.arena.get(L->w64, S->s_nnz);
    copy_d(ctx, L->ptr.p, S->s_ptr.p, (g.n + 1) * sizeof(int32_t));
    copy_d(ctx, L->col.p, S->s_col.p, S->s_nnz * sizeof(int32_t));
    copy_d(ctx, L->w64.p, S->s_w64.p, S->s_nnz * sizeof(double));
    H.arena.get(L->D64, g.n);
    if (with_D) copy_d(ctx, L->D64.p, g.D64.p, g.n * sizeof(double));
    else memset_d(ctx, L->D64.p, 0, g.n * sizeof(double));
    H.arena.get(L->diag64, g.n);
    launch(ctx, k_amg_diag, cdiv(g.n, kBlock), kBlock, 0, g.n, (const int32_t *)L->ptr.p,
           (const double *)L->w64.p, (const double *)L->D64.p, L->diag64.p);
    return L;
}

// aggregate level L into a new coarse level
std::unique_ptr<AmgLevel> coarsen(grass_ctx_t ctx, AmgHier &H, AmgLevel &L) {
    const int64_t n = L.n;
    Arena &tmp = ctx->amg_tmp;        // this level's temporaries
    tmp.reset();
    ASpan<int32_t> mate, cand, anchor, leader, jslot, jcount;
    tmp.get(mate, n);
    tmp.get(cand, n);
    tmp.get(anchor, n);
    tmp.get(leader, n);
    tmp.get(jslot, n);
    tmp.get(jcount, n);
    memset_d(ctx, mate.p, 0xFF, n * sizeof(int32_t));     // -1
    memset_d(ctx, jslot.p, 0xFF, n * sizeof(int32_t));
    // flags[4 + (round & 1)]: round `round` matched something; the next
    // round reads it (no host round trip per round)
    int *chg = ctx->flags.p + 4;
    const int64_t g = cdiv(n, kBlock);
    const int one = 1;
    GCK(cudaMemcpyAsync(chg + 1, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    for (int round = 0; round < kMatchRounds; ++round) {
        int *cur = chg + (round & 1);
        const int *prev = chg + ((round + 1) & 1);
        memset_d(ctx, cur, 0, sizeof(int));
        if (n <= ctx->amg_warp_setup_n)
            launch(ctx, k_amg_cand_w, cdiv(n * 32, kBlock), kBlock, 0, n, (const int32_t *)L.ptr.p,
                   (const int32_t *)L.col.p, (const double *)L.w64.p, (const int32_t *)mate.p, cand.p,
                   prev);
        else
            launch(ctx, k_amg_cand, g, kBlock, 0, n, (const int32_t *)L.ptr.p, (const int32_t *)L.col.p,
                   (const double *)L.w64.p, (const int32_t *)mate.p, cand.p, prev);
        launch(ctx, k_amg_pair, g, kBlock, 0, n, (const int32_t *)cand.p, mate.p, prev, cur);
    }
    launch(ctx, k_amg_join, g, kBlock, 0, n, (const int32_t *)L.ptr.p, (const int32_t *)L.col.p,
           (const double *)L.w64.p, (const int32_t *)mate.p, anchor.p, leader.p);
    launch(ctx, k_amg_slots, g, kBlock, 0, n, (const int32_t *)L.ptr.p, (const int32_t *)L.col.p,
           (const int32_t *)mate.p, (const int32_t *)anchor.p, jslot.p, jcount.p);
    ASpan<int64_t> flag, pos;
    tmp.get(flag, n + 1);
    tmp.get(pos, n + 1);
    launch(ctx, k_amg_leadflag, g, kBlock, 0, n, (const int32_t *)leader.p, flag.p);
    int64_t nc = 0;
    scan_i64(ctx, flag.p, pos.p, n, &nc);
    auto C = std::make_unique<AmgLevel>();
    C->n = nc;
    H.arena.get(L.agg, n);
    ASpan<int64_t> mcnt, moff;
    tmp.get(mcnt, nc + 1);
    tmp.get(moff, nc + 1);
    launch(ctx, k_amg_agg, g, kBlock, 0, n, (const int32_t *)leader.p, (const int64_t *)pos.p,
           (const int32_t *)mate.p, (const int32_t *)jcount.p, L.agg.p, mcnt.p);
    int64_t nm = 0;
    scan_i64(ctx, mcnt.p, moff.p, nc, &nm);
    if (nm != n) fail(GRASS_ERR_CUDA, "multigrid aggregation lost vertices");
    H.arena.get(L.mem, n);
    H.arena.get(L.mptr, nc + 1);
    launch(ctx, k_amg_members, g, kBlock, 0, n, (const int32_t *)leader.p, (const int32_t *)mate.p,
           (const int32_t *)anchor.p, (const int32_t *)jslot.p, (const int32_t *)jcount.p,
           (const int32_t *)L.agg.p, (const int64_t *)moff.p, L.mem.p);
    launch(ctx, k_i64_to_i32, cdiv(nc + 1, kBlock), kBlock, 0, nc + 1, (const int64_t *)moff.p,
           L.mptr.p);
    // coarse matrix
    const int64_t gc = cdiv(nc, kBlock);
    ASpan<int64_t> ccnt, coff;
    tmp.get(ccnt, nc + 1);
    tmp.get(coff, nc + 1);
    const bool wf = n <= ctx->amg_warp_setup_n;
    if (wf)
        launch(ctx, k_amg_ccount_w, cdiv(nc * 32, kBlock), kBlock, 0, nc, (const int32_t *)L.mptr.p,
               (const int32_t *)L.mem.p, (const int32_t *)L.ptr.p, (const int32_t *)L.col.p,
               (const int32_t *)L.agg.p, ccnt.p);
    else
        launch(ctx, k_amg_ccount, gc, kBlock, 0, nc, (const int32_t *)L.mptr.p, (const int32_t *)L.mem.p,
               (const int32_t *)L.ptr.p, (const int32_t *)L.col.p, (const int32_t *)L.agg.p, ccnt.p);
    int64_t cnnz = 0;
    scan_i64(ctx, ccnt.p, coff.p, nc, &cnnz);
    C->nnz = cnnz;
    H.arena.get(C->ptr, nc + 1);
    H.arena.get(C->col, cnnz);
    H.arena.get(C->w64, cnnz);
    H.arena.get(C->D64, nc);
    H.arena.get(C->diag64, nc);
    if (wf)
        launch(ctx, k_amg_cfill_w, cdiv(nc * 32, kBlock), kBlock, 0, nc, (const int32_t *)L.mptr.p,
               (const int32_t *)L.mem.p, (const int32_t *)L.ptr.p, (const int32_t *)L.col.p,
               (const double *)L.w64.p, (const double *)L.D64.p, (const int32_t *)L.agg.p,
               (const int64_t *)coff.p, C->ptr.p, C->col.p, C->w64.p, C->D64.p, C->diag64.p);
    else
        launch(ctx, k_amg_cfill, gc, kBlock, 0, nc, (const int32_t *)L.mptr.p, (const int32_t *)L.mem.p,
               (const int32_t *)L.ptr.p, (const int32_t *)L.col.p, (const double *)L.w64.p,
               (const double *)L.D64.p, (const int32_t *)L.agg.p, (const int64_t *)coff.p, C->ptr.p,
               C->col.p, C->w64.p, C->D64.p, C->diag64.p);
    return C;
}

// aggcol[j] = agg[col[j]]: the coarse vertex of each entry's column
__global__ void k_amg_aggcol(int64_t nnz, const int32_t *col, const int32_t *agg, int32_t *aggcol) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nnz) aggcol[j] = agg[col[j]];
}

__global__ void k_sum_d(int64_t n, const double *D, double *out) {
    // one block: deterministic sum of a small vector
    __shared__ double sh[kBlock];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += D[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

}  // namespace

AmgHier &amg_get(grass_ctx_t ctx, grass_sparsifier_t S, bool with_D) {
    auto &slot = S->amg[with_D ? 1 : 0];
    if (slot) return *slot;
    if (S->is_tree || S->s_nnz == 0) fail(GRASS_ERR_INVALID, "multigrid needs a sparsifier with off-tree edges");
    auto H = std::make_unique<AmgHier>();
    H->lv.push_back(level0(ctx, *H, S, with_D));
    while (H->lv.back()->n > kCoarse) {
        if ((int)H->lv.size() >= kMaxLevels) fail(GRASS_ERR_CUDA, "multigrid: too many levels");
        auto C = coarsen(ctx, *H, *H->lv.back());
        if (C->n > H->lv.back()->n * 95 / 100)
            fail(GRASS_ERR_CUDA, "multigrid coarsening stalled at " + std::to_string(C->n) + " vertices");
        H->lv.push_back(std::move(C));
    }
    // FP32 copies and V-cycle vectors
    for (size_t l = 0; l < H->lv.size(); ++l) {
        AmgLevel &L = *H->lv[l];
        H->arena.get(L.w32, std::max<int64_t>(L.nnz, 1));
        H->arena.get(L.diag32, L.n);
        launch(ctx, k_amg_f32, cdiv(L.nnz, kBlock), kBlock, 0, L.nnz, (const double *)L.w64.p, L.w32.p);
        launch(ctx, k_amg_f32, cdiv(L.n, kBlock), kBlock, 0, L.n, (const double *)L.diag64.p,
               L.diag32.p);
        if (l > 0) {
            H->arena.get(L.vb, L.n * sizeof(double) + 256);
            H->arena.get(L.vx, L.n * sizeof(double) + 256);
        }
        H->arena.get(L.vt, L.n * sizeof(double) + 256);
        if (l + 1 < H->lv.size()) {
            H->arena.get(L.aggcol, std::max<int64_t>(L.nnz, 1));
            launch(ctx, k_amg_aggcol, cdiv(L.nnz, kBlock), kBlock, 0, L.nnz, (const int32_t *)L.col.p,
                   (const int32_t *)L.agg.p, L.aggcol.p);
        }
    }
    // coarsest: dense (grounded) inverse
    AmgLevel &Lc = *H->lv.back();
    H->nc = Lc.n;
    double *dsum = ctx->scal.p + DS_RED + 51;
    launch(ctx, k_sum_d, 1, kBlock, 0, Lc.n, (const double *)Lc.D64.p, dsum);
    double ds = 0.0;
    d2h(ctx, &ds, dsum, sizeof(double));
    H->singular = !(ds > 0.0);
    H->cinv64.alloc(Lc.n * Lc.n);
    H->cinv32.alloc(Lc.n * Lc.n);
    memset_d(ctx, H->cinv64.p, 0, Lc.n * Lc.n * sizeof(double));
    launch(ctx, k_amg_dense, cdiv(Lc.n, kBlock), kBlock, 0, Lc.n, (const int32_t *)Lc.ptr.p,
           (const int32_t *)Lc.col.p, (const double *)Lc.w64.p, (const double *)Lc.diag64.p,
           H->singular ? 1 : 0, H->cinv64.p);
    if (ctx->num_sms > 0 && Lc.n > 1) {
        // across the grid (cooperative): nc steps, one barrier each
        ctx->amg_tmp.reset();
        ASpan<double> other;
        ctx->amg_tmp.get(other, Lc.n * Lc.n);
        const int grid = (int)std::min<int64_t>(Lc.n, coop_grid(ctx, k_amg_gj_grid, 256, 0, Lc.n * 256));
        int64_t nc = Lc.n;
        double *m0 = H->cinv64.p, *m1 = other.p;
        unsigned int *bar = ctx->gbar.p;
        long long budget = ctx->wait_budget;
        int *err = ctx->flags.p + 3;
        GCK(cudaMemsetAsync(bar, 0, sizeof(unsigned int), ctx->stream));
        void *args[] = {&nc, &m0, &m1, &bar, &budget, &err};
        GCK(cudaLaunchCooperativeKernel((const void *)k_amg_gj_grid, dim3(grid), dim3(256), args, 0,
                                        ctx->stream));
        ctx->launches++;
        // the last step (p = nc - 1) wrote M1 when nc - 1 is even
        if (((nc - 1) & 1) == 0) copy_d(ctx, H->cinv64.p, other.p, nc * nc * sizeof(double));
        if (H->singular) launch(ctx, k_amg_ground_inv, 1, 256, 0, nc, H->cinv64.p);
        ctx->sync();
        check_timeout(ctx);
    } else {
        launch(ctx, k_amg_gauss_jordan, 1, 1024, 0, Lc.n, H->cinv64.p, H->singular ? 1 : 0);
    }
    launch(ctx, k_amg_f32, cdiv(Lc.n * Lc.n, kBlock), kBlock, 0, Lc.n * Lc.n,
           (const double *)H->cinv64.p, H->cinv32.p);
    ctx->sync();
    // keep up to 256 MB of temporaries for the next hierarchy
    if (ctx->amg_tmp.bytes() > ((size_t)256 << 20)) ctx->amg_tmp = Arena();
    slot = std::move(H);
    return *slot;
}

// ---------------------------------------------------------------- V-cycle

template <typename T>
static void vcycle_T(grass_ctx_t ctx, AmgHier &H, size_t l, const T *b, T *x, int nu) {
    AmgLevel &L = *H.lv[l];
    const int64_t n = L.n;
    const int64_t g = cdiv(n, kBlock);
    if (l + 1 == H.lv.size()) {
        const T *ci;
        if constexpr (sizeof(T) == 8) ci = H.cinv64.p;
        else ci = H.cinv32.p;
        launch(ctx, k_coarse_apply<T>, 1, kBlock, 0, n, ci, b, x);
        return;
    }
    const int32_t *ptr = L.ptr.p, *col = L.col.p;
    const T *w = lvl_w<T>(L), *diag = lvl_diag<T>(L);
    // the sweeps alternate between x and t; `cur` holds the iterate.  With
    // nu sweeps before and nu after (2 nu in all, an even count) the last
    // one ends in x.
    T *t = reinterpret_cast<T *>(L.vt.p);
    T *cur = x, *nxt = t;
    launch(ctx, k_jac0<T>, g, kBlock, 0, n, b, diag, cur);           // pre-smoothing from 0
    for (int s = 1; s < nu; ++s) {
        launch(ctx, k_jac<T>, g, kBlock, 0, n, ptr, col, w, diag, b, (const T *)cur, nxt);
        std::swap(cur, nxt);
    }
    AmgLevel &C = *H.lv[l + 1];
    T *bc = reinterpret_cast<T *>(C.vb.p), *xc = reinterpret_cast<T *>(C.vx.p);
    launch(ctx, k_residual<T>, g, kBlock, 0, n, ptr, col, w, diag, b, (const T *)cur, nxt);
    launch(ctx, k_restrict<T>, cdiv(C.n, kBlock), kBlock, 0, C.n, (const int32_t *)L.mptr.p,
           (const int32_t *)L.mem.p, (const T *)nxt, bc);
    vcycle_T<T>(ctx, H, l + 1, bc, xc, nu);
    launch(ctx, k_prolong<T>, g, kBlock, 0, n, (const int32_t *)L.agg.p, (const T *)xc, cur);
    for (int s = 0; s < nu; ++s) {
        launch(ctx, k_jac<T>, g, kBlock, 0, n, ptr, col, w, diag, b, (const T *)cur, nxt);
        std::swap(cur, nxt);
    }
    if (cur != x) copy_d(ctx, x, cur, n * sizeof(T));
}

void amg_vcycle(grass_ctx_t ctx, grass_sparsifier_t S, bool with_D, grass_prec prec, const void *r,
                void *z) {
    AmgHier &H = amg_get(ctx, S, with_D);
    if (prec == GRASS_FP64) vcycle_T<double>(ctx, H, 0, (const double *)r, (double *)z, ctx->amg_sweeps);
    else vcycle_T<float>(ctx, H, 0, (const float *)r, (float *)z, ctx->amg_sweeps);
}

// ---------------------------------------------------------------- PCG on A with the V-cycle
// Device scalars s: [0] r.z, [1] p.q, [2] r.r, [3] new r.z, [4] go (1 while
// the iteration goes on), [5] iterations done.  Every kernel of an
// iteration reads `go`, so iterations replayed after convergence change
// nothing.

template <typename T>
__global__ void k_ap_axpy(int64_t n, const double *s, T *x, T *r, const T *p, const T *q) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || s[4] == 0.0) return;
    const T a = (T)(s[0] / s[1]);
    x[i] += a * p[i];
    r[i] -= a * q[i];
}

// one thread: count the iteration just done and decide whether to go on
__global__ void k_ap_check(double *s, double tol2, double maxit) {
    if (s[4] == 0.0) return;
    s[5] += 1.0;
    if (!(s[2] > tol2) || s[5] >= maxit) s[4] = 0.0;
}

template <typename T>
__global__ void k_ap_p(int64_t n, const double *s, const T *z, T *p) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || s[4] == 0.0) return;
    p[i] = z[i] + (T)(s[3] / s[0]) * p[i];
}

__global__ void k_ap_shift(double *s) {
    if (s[4] != 0.0) s[0] = s[3];
}

__global__ void k_ap_init(double *s, double tol2) {
    s[4] = s[2] > tol2 ? 1.0 : 0.0;
    s[5] = 0.0;
}

template <typename T>
int amg_pcg(grass_ctx_t ctx, grass_sparsifier_t S, const T *rhs, T *e, double tol_abs, int maxit) {
    const GraphData &g = S->tree->g;
    const int64_t n = g.n, gn = cdiv(n, kBlock);
    const grass_prec prec = sizeof(T) == 8 ? GRASS_FP64 : GRASS_FP32;
    AmgHier &H = amg_get(ctx, S, true);
    if (ctx->amg_fused && ctx->num_sms > 0 && ctx->amg_sweeps == 1 &&
        (int)H.lv.size() <= kAmgFusedLevels)
        return amg_pcg_fused<T>(ctx, S, H, rhs, e, tol_abs, maxit);
    T *r = ctx->scr<T>(SCR_PCG_R, n);
    T *z = ctx->scr<T>(SCR_PCG_Z, n);
    T *p = ctx->scr<T>(SCR_PCG_P, n);
    T *q = ctx->scr<T>(SCR_PCG_Q, n);
    double *s = ctx->scal.p + DS_RED + 24;        // [24 .. 29]
    const void *wA = prec == GRASS_FP64 ? (const void *)g.adj_w64.p : (const void *)g.adj_w32.p;
    const void *DA = prec == GRASS_FP64 ? (const void *)g.D64.p : (const void *)g.D32.p;
    const double tol2 = tol_abs * tol_abs;
    // the work runs on the context's capture stream, after the caller's work
    if (!ctx->cap_stream) {
        GCK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        GCK(cudaEventCreateWithFlags(&ctx->cap_ev[0], cudaEventDisableTiming));
        GCK(cudaEventCreateWithFlags(&ctx->cap_ev[1], cudaEventDisableTiming));
    }
    cudaStream_t user = ctx->stream;
    const bool own = ctx->tfam == 0;              // kernel timing records events on the caller's stream
    if (own) {
        GCK(cudaEventRecord(ctx->cap_ev[0], user));
        GCK(cudaStreamWaitEvent(ctx->cap_stream, ctx->cap_ev[0], 0));
        ctx->stream = ctx->cap_stream;
    }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto iteration = [&]() {
        lap_mm(ctx, 1, prec, n, 2 * g.m, g.adj_ptr.p, g.adj_col.p, wA, DA, p, q, nullptr,
               GRASS_KF_SPMM_G, &g.heavy);
        dot_cols(ctx, 1, prec, n, p, q, s + 1);
        launch(ctx, k_ap_axpy<T>, gn, kBlock, 0, n, (const double *)s, e, r, (const T *)p, (const T *)q);
        dot_cols(ctx, 1, prec, n, r, r, s + 2);
        launch(ctx, k_ap_check, 1, 1, 0, s, tol2, (double)maxit);
        amg_vcycle(ctx, S, true, prec, r, z);
        dot_cols(ctx, 1, prec, n, r, z, s + 3);
        launch(ctx, k_ap_p<T>, gn, kBlock, 0, n, (const double *)s, (const T *)z, p);
        launch(ctx, k_ap_shift, 1, 1, 0, s);
    };
    double st[2] = {0.0, 0.0};
    try {
        memset_d(ctx, e, 0, n * sizeof(T));
        copy_d(ctx, r, rhs, n * sizeof(T));
        dot_cols(ctx, 1, prec, n, r, r, s + 2);
        launch(ctx, k_ap_init, 1, 1, 0, s, tol2);
        amg_vcycle(ctx, S, true, prec, r, z);
        copy_d(ctx, p, z, n * sizeof(T));
        dot_cols(ctx, 1, prec, n, r, z, s);
        d2h(ctx, st, s + 4, sizeof(st));
        if (st[0] != 0.0 && maxit > 0) {
            iteration();                          // plain: fills the shape caches
            bool captured = false;
            int64_t per = 0;
            if (own) {
                const int64_t l0 = ctx->launches;
                if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                    bool ok = true;
                    try {
                        iteration();
                    } catch (...) {
                        ok = false;
                    }
                    cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
                    captured = ok && ce == cudaSuccess && graph &&
                               cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
                    if (!captured) cudaGetLastError();
                } else {
                    cudaGetLastError();
                }
                per = ctx->launches - l0;
                ctx->launches = l0;
            }
            constexpr int kCheck = 8;
            d2h(ctx, st, s + 4, sizeof(st));
            while (st[0] != 0.0) {
                for (int j = 0; j < kCheck; ++j) {
                    if (captured) {
                        GCK(cudaGraphLaunch(exec, ctx->stream));
                        ctx->launches += per;
                    } else {
                        iteration();
                    }
                }
                d2h(ctx, st, s + 4, sizeof(st));
            }
        }
    } catch (...) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (own) {
            ctx->stream = user;
            cudaEventRecord(ctx->cap_ev[1], ctx->cap_stream);
            cudaStreamWaitEvent(user, ctx->cap_ev[1], 0);
        }
        throw;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (own) {
        ctx->stream = user;
        GCK(cudaEventRecord(ctx->cap_ev[1], ctx->cap_stream));
        GCK(cudaStreamWaitEvent(user, ctx->cap_ev[1], 0));
    }
    return (int)st[1];
}

template int amg_pcg<double>(grass_ctx_t, grass_sparsifier_t, const double *, double *, double, int);
template int amg_pcg<float>(grass_ctx_t, grass_sparsifier_t, const float *, float *, double, int);

// ---------------------------------------------------------------- CG on L_S

__global__ void k_amg_center(int64_t n, double *y, const double *sum) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] -= *sum / (double)n;
}

__global__ void k_amg_ones(int64_t n, double *o) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = 1.0;
}

// x += a p, r -= a q (a = num / den)
__global__ void k_amg_axpy(int64_t n, const double *num, const double *den, double *x, double *r,
                           const double *p, const double *q) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = *num / *den;
    x[i] += a * p[i];
    r[i] -= a * q[i];
}

// p = z + (num / den) p
__global__ void k_amg_p(int64_t n, const double *num, const double *den, const double *z, double *p) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = z[i] + (*num / *den) * p[i];
}

int amg_cg_lap(grass_ctx_t ctx, grass_sparsifier_t S, const double *y, double *x, double tol,
               int maxit) {
    const int64_t n = S->tree->g.n;
    const int64_t g = cdiv(n, kBlock);
    amg_get(ctx, S, false);
    double *r = ctx->scr<double>(SCR_PART_X, n);
    double *z = ctx->scr<double>(SCR_PART_Y, n);
    double *p = ctx->scr<double>(SCR_PART_1, n);
    double *q = ctx->scr<double>(SCR_SIM_E, n);
    double *ones = ctx->scr<double>(SCR_TMP3, n);
    double *sc = ctx->scal.p + DS_RED + 52;     // [52..57] scalars of this solve
    launch(ctx, k_amg_ones, g, kBlock, 0, n, ones);
    copy_d(ctx, r, y, n * sizeof(double));
    dot_cols(ctx, 1, GRASS_FP64, n, r, ones, sc);
    launch(ctx, k_amg_center, g, kBlock, 0, n, r, (const double *)sc);
    memset_d(ctx, x, 0, n * sizeof(double));
    dot_cols(ctx, 1, GRASS_FP64, n, r, r, sc + 1);       // ||y||^2
    double yy = 0.0;
    d2h(ctx, &yy, sc + 1, sizeof(double));
    if (!(yy > 0.0)) return 0;
    amg_vcycle(ctx, S, false, GRASS_FP64, r, z);
    copy_d(ctx, p, z, n * sizeof(double));
    dot_cols(ctx, 1, GRASS_FP64, n, r, z, sc + 2);       // r.z
    const void *w = S->s_w64.p;
    int k = 0;
    for (; k < maxit; ++k) {
        lap_mm(ctx, 1, GRASS_FP64, n, S->s_nnz, S->s_ptr.p, S->s_col.p, w, nullptr, p, q, nullptr,
               GRASS_KF_SPMM_S, &S->s_heavy);
        dot_cols(ctx, 1, GRASS_FP64, n, p, q, sc + 3);
        launch(ctx, k_amg_axpy, g, kBlock, 0, n, (const double *)(sc + 2), (const double *)(sc + 3),
               x, r, (const double *)p, (const double *)q);
        dot_cols(ctx, 1, GRASS_FP64, n, r, r, sc + 4);
        double rr = 0.0;
        d2h(ctx, &rr, sc + 4, sizeof(double));
        if (std::sqrt(rr) <= tol * std::sqrt(yy)) {
            ++k;
            break;
        }
        amg_vcycle(ctx, S, false, GRASS_FP64, r, z);
        dot_cols(ctx, 1, GRASS_FP64, n, r, z, sc + 5);
        launch(ctx, k_amg_p, g, kBlock, 0, n, (const double *)(sc + 5), (const double *)(sc + 2),
               (const double *)z, p);
        copy_d(ctx, sc + 2, sc + 5, sizeof(double));
    }
    return k;
}

}  // namespace grass
