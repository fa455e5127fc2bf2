// batch.cu -- the batched form: many independent graphs sparsified and
// solved together as one block-diagonal matrix (grass_build_forest).
//
// Everything that is per vertex or per edge (SpMM, the forest solve, the
// heat of every off-sparsifier edge) runs over the whole batch in the same
// launches as for one graph.  What the method defines per graph -- lambda_min
// and lambda_max (Sec. IV-C), theta_sigma and heat_max (Eq.
// heatratio_final), the PCG scalars (Sec. V-A) -- is reduced per graph over
// "chunks": ranges of rows or edges that never cross a graph boundary and
// whose length depends only on the graph itself.  Each reduction sums a
// chunk in a fixed order and then a graph's chunks in a fixed order, so a
// graph's results do not depend on which other graphs share the batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace grass {
namespace {

constexpr int kBT = 256;                  // threads of the chunked kernels
constexpr int64_t kRowChunk = 4096;       // rows per chunk (PCG vectors, lambda_min)
constexpr int64_t kEdgeChunk = 8192;      // edges per chunk (quadratic forms, heat)

// Ranges [beg[c], beg[c+1]) tiling [0, total) per graph: chunk c belongs to
// graph seg[c]; graph k owns chunks [first[k], first[k+1]).
struct Chunks {
    int64_t count = 0;
    DBuf<int64_t> beg;
    DBuf<int32_t> seg, first;

    void build(grass_ctx_t ctx, const std::vector<int64_t> &off, int64_t len) {
        const int64_t G = (int64_t)off.size() - 1;
        std::vector<int64_t> b;
        std::vector<int32_t> s, f(G + 1);
        for (int64_t k = 0; k < G; ++k) {
            f[k] = (int32_t)b.size();
            for (int64_t x = off[k]; x < off[k + 1]; x += len) {
                b.push_back(x);
                s.push_back((int32_t)k);
            }
        }
        f[G] = (int32_t)b.size();
        b.push_back(off[G]);
        count = (int64_t)s.size();
        beg.alloc(b.size());
        seg.alloc(std::max<size_t>(s.size(), 1));
        first.alloc(f.size());
        h2d(ctx, beg.p, b.data(), b.size() * sizeof(int64_t));
        if (!s.empty()) h2d(ctx, seg.p, s.data(), s.size() * sizeof(int32_t));
        h2d(ctx, first.p, f.data(), f.size() * sizeof(int32_t));
    }
};

template <typename T>
__device__ inline T block_sum(T v, T *sh) {
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    return s;   // valid in thread 0
}

// Sums over each graph's chunks, K values per chunk: out[j*G + k] (value j
// of graph k).  One warp per graph, lanes stride over its chunks, fixed xor
// tree.
__global__ void k_b_sum(int64_t G, int K, const int32_t *first, const double *part, double *out) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= G) return;
    for (int j = 0; j < K; ++j) {
        double s = 0.0;
        for (int64_t c = first[k] + lane; c < first[k + 1]; c += 32) s += part[c * K + j];
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) out[(int64_t)j * G + k] = s;
    }
}

// ---------------------------------------------------------------- per-graph estimates

// lambda_min per graph (Sec. IV-C-2): min over the graph's rows of
// L_G(p,p) / L_S(p,p); a block per row chunk, then one atomicMin on the bit
// pattern of a positive double (order-free).
__global__ void k_b_lmin(const int64_t *cbeg, const int32_t *cseg, const double *degG,
                         const double *degS, unsigned long long *out) {
    __shared__ double sh[32];
    const int64_t c = blockIdx.x;
    double mn = 1.0 / 0.0;
    for (int64_t p = cbeg[c] + threadIdx.x; p < cbeg[c + 1]; p += blockDim.x)
        mn = fmin(mn, degG[p] / degS[p]);
    for (int d = 16; d > 0; d >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, d));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = mn;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mn = fmin(mn, sh[w]);
        atomicMin(out + cseg[c], (unsigned long long)__double_as_longlong(mn));
    }
}

// Rayleigh quotient parts per edge chunk (Sec. IV-C-1, Eq. 2):
// part[2c] = sum_e w_e (x_u - x_v)^2 over all edges, part[2c+1] over S.
template <typename T>
__global__ void k_b_quad(const int64_t *cbeg, const int32_t *eu, const int32_t *ev,
                         const double *ew, const uint8_t *in_s, const T *x, double *part) {
    __shared__ double sh[32];
    const int64_t c = blockIdx.x;
    double g = 0.0, s = 0.0;
    for (int64_t e = cbeg[c] + threadIdx.x; e < cbeg[c + 1]; e += blockDim.x) {
        double d = (double)x[eu[e]] - (double)x[ev[e]];
        double h = ew[e] * d * d;
        g += h;
        if (in_s[e]) s += h;
    }
    g = block_sum(g, sh);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        part[2 * c] = g;
        part[2 * c + 1] = s;
    }
}

// heat_max per graph over its off-sparsifier edges (order-free atomicMax)
template <typename T>
__global__ void k_b_hmax(const int64_t *cbeg, const int32_t *cseg, const T *heat,
                         unsigned long long *out) {
    __shared__ double sh[32];
    const int64_t c = blockIdx.x;
    double mx = 0.0;
    for (int64_t i = cbeg[c] + threadIdx.x; i < cbeg[c + 1]; i += blockDim.x)
        mx = fmax(mx, (double)heat[i]);
    for (int d = 16; d > 0; d >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, d));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, sh[w]);
        atomicMax(out + cseg[c], (unsigned long long)__double_as_longlong(mx));
    }
}

// filter (Eq. heatratio_final) with the threshold of each edge's graph
template <typename T>
__global__ void k_b_flag(const int64_t *cbeg, const int32_t *cseg, const T *heat,
                         const double *thr, int64_t *flag) {
    const int64_t c = blockIdx.x;
    const double t = thr[cseg[c]];
    for (int64_t i = cbeg[c] + threadIdx.x; i < cbeg[c + 1]; i += blockDim.x)
        flag[i] = (double)heat[i] >= t ? 1 : 0;
}

__global__ void k_b_scatter(int64_t moff, const int64_t *flag, const int64_t *pos,
                            const int32_t *off_eid, int64_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < moff && flag[i]) out[pos[i]] = off_eid[i];
}

// first off-sparsifier edge of every graph: lower bound of its first edge id
__global__ void k_b_lower(int64_t G, const int64_t *eoff, int64_t moff, const int32_t *off_eid,
                          int64_t *out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k > G) return;
    int64_t lo = 0, hi = moff, key = eoff[k];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)off_eid[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    out[k] = lo;
}

__global__ void k_bits_init(int64_t G, unsigned long long *a, unsigned long long v) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < G) a[k] = v;
}

std::vector<int64_t> offtree_offsets(grass_ctx_t ctx, grass_sparsifier_t S) {
    const GraphData &g = S->tree->g;
    const int64_t G = g.nseg;
    DBuf<int64_t> eo, out;
    eo.alloc(G + 1);
    out.alloc(G + 1);
    h2d(ctx, eo.p, g.seg_eoff.data(), (G + 1) * sizeof(int64_t));
    launch(ctx, k_b_lower, cdiv(G + 1, kBT), kBT, 0, G, (const int64_t *)eo.p, S->m_off,
           (const int32_t *)S->off_eid.p, out.p);
    std::vector<int64_t> h(G + 1);
    d2h(ctx, h.data(), out.p, (G + 1) * sizeof(int64_t));
    return h;
}

// ---------------------------------------------------------------- batched PCG (Sec. V-A)

enum { BS_BB = 0, BS_RR, BS_RZ, BS_PQ, BS_ALPHA, BS_RZN, BS_RZO, BS_BETA, BS_IT, BS_RES,
       BS_IRZ, BS_IPQ, BS_IALPHA, BS_IRZN, BS_IBETA, BS_TOL, BS_BN, BS_BN2, BS_N };

template <typename T>
struct BMat {
    const int32_t *ptr, *col;
    const T *w, *D;
};

// Q = (L + D) P on the rows of each active graph; part[c] = P.Q over the chunk
template <typename T>
__global__ void k_b_matvec(const int64_t *cbeg, const int32_t *cseg, const int *act, BMat<T> A,
                           const T *P, T *Q, double *part) {
    __shared__ double sh[32];
    const int64_t c = blockIdx.x;
    if (!act[cseg[c]]) {
        if (threadIdx.x == 0) part[c] = 0.0;
        return;
    }
    Acc<T> ac;
    for (int64_t i = cbeg[c] + threadIdx.x; i < cbeg[c + 1]; i += blockDim.x) {
        const T pi = P[i];
        T q = A.D ? A.D[i] * pi : (T)0;
        for (int32_t j = A.ptr[i]; j < A.ptr[i + 1]; ++j) q += A.w[j] * (pi - P[A.col[j]]);
        Q[i] = q;
        ac.add_prod(pi, q);
    }
    const double acc = block_sum(ac.value(), sh);
    if (threadIdx.x == 0) part[c] = acc;
}

// X += alpha P, R -= alpha Q, Z = R; part[c] = R.R   (per-graph alpha)
template <typename T>
__global__ void k_b_update(const int64_t *cbeg, const int32_t *cseg, const int *act,
                           const double *alpha, T *X, const T *P, T *R, const T *Q, T *Z,
                           double *part) {
    __shared__ double sh[32];
    const int64_t c = blockIdx.x;
    const int k = cseg[c];
    if (!act[k]) {
        if (threadIdx.x == 0) part[c] = 0.0;
        return;
    }
    const T a = (T)alpha[k];
    Acc<T> ac;
    for (int64_t i = cbeg[c] + threadIdx.x; i < cbeg[c + 1]; i += blockDim.x) {
        X[i] += a * P[i];
        T r = R[i] - a * Q[i];
        R[i] = r;
        Z[i] = r;
        ac.add_prod(r, r);
    }
    const double acc = block_sum(ac.value(), sh);
    if (threadIdx.x == 0) part[c] = acc;
}

// part[2c] = R.Z, part[2c+1] = R.Zold
template <typename T>
__global__ void k_b_dot2(const int64_t *cbeg, const int32_t *cseg, const int *act, const T *R,
                         const T *Z, const T *Zo, double *part) {
    __shared__ double sh[32];
    const int64_t c = blockIdx.x;
    if (!act[cseg[c]]) {
        if (threadIdx.x == 0) part[2 * c] = part[2 * c + 1] = 0.0;
        return;
    }
    Acc<T> aa, ab;
    for (int64_t i = cbeg[c] + threadIdx.x; i < cbeg[c + 1]; i += blockDim.x) {
        const T r = R[i];
        aa.add_prod(r, Z[i]);
        if (Zo) ab.add_prod(r, Zo[i]);
    }
    const double a = block_sum(aa.value(), sh);
    const double b = block_sum(ab.value(), sh);
    if (threadIdx.x == 0) {
        part[2 * c] = a;
        part[2 * c + 1] = b;
    }
}

// P = Z + beta P; Zold = Z (when given)
template <typename T>
__global__ void k_b_pupd(const int64_t *cbeg, const int32_t *cseg, const int *act,
                         const double *beta, const T *Z, T *P, T *Zo) {
    const int64_t c = blockIdx.x;
    const int k = cseg[c];
    if (!act[k]) return;
    const T b = (T)beta[k];
    for (int64_t i = cbeg[c] + threadIdx.x; i < cbeg[c + 1]; i += blockDim.x) {
        const T z = Z[i];
        P[i] = z + b * P[i];
        if (Zo) Zo[i] = z;
    }
}

template <typename T>
__global__ void k_b_start(int64_t n, const double *b, T *R, T *X, T *Zi) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    R[i] = (T)b[i];
    X[i] = (T)0;
    if (Zi) Zi[i] = (T)0;
}

template <typename T>
__global__ void k_b_copy_act(const int64_t *cbeg, const int32_t *cseg, const int *act, const T *A,
                             T *B, T *Zero) {
    const int64_t c = blockIdx.x;
    if (!act[cseg[c]]) return;
    for (int64_t i = cbeg[c] + threadIdx.x; i < cbeg[c + 1]; i += blockDim.x) {
        B[i] = A[i];
        if (Zero) Zero[i] = (T)0;
    }
}

// r = b - (L_G + D) x in FP64 (FP64 matrix and iterate); part[c] = r.r
__global__ void k_b_resid(const int64_t *cbeg, const int32_t *ptr, const int32_t *col,
                          const double *w, const double *D, const double *x, const double *b,
                          double *r, double *part) {
    __shared__ double sh[32];
    const int64_t c = blockIdx.x;
    double acc = 0.0;
    for (int64_t i = cbeg[c] + threadIdx.x; i < cbeg[c + 1]; i += blockDim.x) {
        const double xi = x[i];
        double q = D[i] * xi;
        for (int32_t j = ptr[i]; j < ptr[i + 1]; ++j) q += w[j] * (xi - x[col[j]]);
        const double ri = b[i] - q;
        r[i] = ri;
        acc += ri * ri;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[c] = acc;
}

// start of a refinement pass for the graphs in it: R = r (in T), X = 0
template <typename T>
__global__ void k_b_pass(const int64_t *cbeg, const int32_t *cseg, const int *inpass,
                         const double *r, T *R, T *X) {
    const int64_t c = blockIdx.x;
    if (!inpass[cseg[c]]) return;
    for (int64_t i = cbeg[c] + threadIdx.x; i < cbeg[c + 1]; i += blockDim.x) {
        R[i] = (T)r[i];
        X[i] = (T)0;
    }
}

// x += X (FP64) for the graphs of the pass
template <typename T>
__global__ void k_b_accum(const int64_t *cbeg, const int32_t *cseg, const int *inpass, const T *X,
                          double *x) {
    const int64_t c = blockIdx.x;
    if (!inpass[cseg[c]]) return;
    for (int64_t i = cbeg[c] + threadIdx.x; i < cbeg[c + 1]; i += blockDim.x) x[i] += (double)X[i];
}

// ---- per-graph scalar steps (one thread per graph)

__global__ void k_bs_init(int64_t G, double *sc, int *act, const int *inpass) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G) return;
    double bb = sc[BS_BB * G + k];
    sc[BS_RR * G + k] = bb;
    sc[BS_IT * G + k] = 0.0;
    act[k] = inpass[k] && bb > 0.0 ? 1 : 0;
}

// alpha = rz / pq; a pq that is not positive gives alpha = 0 and, for the
// outer iteration (stop != 0), ends that graph's iteration
__global__ void k_bs_alpha(int64_t G, int slot_rz, int slot_pq, int slot_alpha, double *sc,
                           int *act, int stop) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G || !act[k]) return;
    double pq = sc[slot_pq * G + k];
    if (!(pq > 0.0)) {
        sc[slot_alpha * G + k] = 0.0;
        if (stop) act[k] = 0;
        return;
    }
    sc[slot_alpha * G + k] = sc[slot_rz * G + k] / pq;
}

// after the update: count the iteration; a graph stops once ||r|| <= tol_k
// ||rhs|| (its tolerance for this pass) or its iteration budget is spent
__global__ void k_bs_check(int64_t G, int maxit, double *sc, int *act, int *nact) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G || !act[k]) return;
    double it = sc[BS_IT * G + k] + 1.0;
    sc[BS_IT * G + k] = it;
    bool go = sqrt(sc[BS_RR * G + k]) > sc[BS_TOL * G + k] * sqrt(sc[BS_BB * G + k]) &&
              it < (double)maxit;
    act[k] = go ? 1 : 0;
    if (go) atomicAdd(nact, 1);
}

// flexible beta = r.(z - z_old) / rz, then rz = r.z  (slot_rzo < 0: plain r.z / rz)
__global__ void k_bs_beta(int64_t G, int slot_rzn, int slot_rzo, int slot_rz, int slot_beta,
                          double *sc, const int *act) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G || !act[k]) return;
    double rzn = sc[slot_rzn * G + k];
    double num = slot_rzo >= 0 ? rzn - sc[slot_rzo * G + k] : rzn;
    double rz = sc[slot_rz * G + k];
    sc[slot_beta * G + k] = rz != 0.0 ? num / rz : 0.0;
    sc[slot_rz * G + k] = rzn;
}

struct BatchPCG {
    grass_ctx_t ctx;
    grass_sparsifier_t S;
    grass_prec prec;
    int64_t n, G;
    Chunks ch;
    DBuf<double> part, sc;
    DBuf<int> act, nact, inpass;
    int inner;
    double tol;
    int maxit;

    double *slot(int s) { return sc.p + (int64_t)s * G; }
    void sum(int K, int s) {
        launch(ctx, k_b_sum, cdiv(G * 32, kBT), kBT, 0, G, K, (const int32_t *)ch.first.p,
               (const double *)part.p, slot(s));
    }
    int64_t sgrid() const { return cdiv(G, kBT); }
};

template <typename T>
struct BVecs {
    T *X, *R, *Z, *Zo, *P, *Q;           // outer
    T *Zi, *Ri, *Wi, *Pi, *Qi;           // inner (sparsifier CG)
};

// z = M^{-1} r with M = L_S + D: the forest solve, then `inner` CG steps on
// L_S + D preconditioned by it (the first step only rescales the forest
// solve).  Z holds r on entry and z on return.
template <typename T>
void b_precond(BatchPCG &B, BVecs<T> &v, const BMat<T> &MS) {
    grass_ctx_t ctx = B.ctx;
    grass_tree_t Tr = B.S->tree;
    const int64_t nc = B.ch.count;
    const int *act = B.act.p;
    const int64_t *cb = B.ch.beg.p;
    const int32_t *cs = B.ch.seg.p;
    if (B.inner <= 0 || B.S->is_tree) {
        tree_solve_inplace(ctx, Tr, Tr->sdd, 1, B.prec, v.Z, nullptr);
        return;
    }
    // Ri = r, Zi = 0, Wi = T^{-1} r, Pi = Wi, irz = Ri.Wi
    launch(ctx, k_b_copy_act<T>, nc, kBT, 0, cb, cs, act, (const T *)v.Z, v.Ri, v.Zi);
    launch(ctx, k_b_copy_act<T>, nc, kBT, 0, cb, cs, act, (const T *)v.Z, v.Wi, (T *)nullptr);
    tree_solve_inplace(ctx, Tr, Tr->sdd, 1, B.prec, v.Wi, nullptr);
    launch(ctx, k_b_copy_act<T>, nc, kBT, 0, cb, cs, act, (const T *)v.Wi, v.Pi, (T *)nullptr);
    launch(ctx, k_b_dot2<T>, nc, kBT, 0, cb, cs, act, (const T *)v.Ri, (const T *)v.Wi,
           (const T *)nullptr, B.part.p);
    B.sum(2, BS_IRZN);
    // irz = irzn (first product): reuse the beta step with no old term
    launch(ctx, k_bs_beta, B.sgrid(), kBT, 0, B.G, BS_IRZN, -1, BS_IRZ, BS_IBETA, B.sc.p, act);
    for (int j = 0; j < B.inner; ++j) {
        launch(ctx, k_b_matvec<T>, nc, kBT, 0, cb, cs, act, MS, (const T *)v.Pi, v.Qi, B.part.p);
        B.sum(1, BS_IPQ);
        launch(ctx, k_bs_alpha, B.sgrid(), kBT, 0, B.G, (int)BS_IRZ, (int)BS_IPQ, (int)BS_IALPHA,
               B.sc.p, B.act.p, 0);
        // Zi += a Pi, Ri -= a Qi, Wi = Ri
        launch(ctx, k_b_update<T>, nc, kBT, 0, cb, cs, act, (const double *)B.slot(BS_IALPHA),
               v.Zi, (const T *)v.Pi, v.Ri, (const T *)v.Qi, v.Wi, B.part.p);
        if (j + 1 == B.inner) break;
        tree_solve_inplace(ctx, Tr, Tr->sdd, 1, B.prec, v.Wi, nullptr);
        launch(ctx, k_b_dot2<T>, nc, kBT, 0, cb, cs, act, (const T *)v.Ri, (const T *)v.Wi,
               (const T *)nullptr, B.part.p);
        B.sum(2, BS_IRZN);
        launch(ctx, k_bs_beta, B.sgrid(), kBT, 0, B.G, BS_IRZN, -1, BS_IRZ, BS_IBETA, B.sc.p, act);
        launch(ctx, k_b_pupd<T>, nc, kBT, 0, cb, cs, act, (const double *)B.slot(BS_IBETA),
               (const T *)v.Wi, v.Pi, (T *)nullptr);
    }
    launch(ctx, k_b_copy_act<T>, nc, kBT, 0, cb, cs, act, (const T *)v.Zi, v.Z, (T *)nullptr);
}

// PCG passes with FP64 iterative refinement: each pass solves A e = r for
// the graphs whose FP64 residual r = b - A x still misses the tolerance
// (vectors in T, scalars FP64), then x += e in FP64.  With FP64 vectors the
// first pass normally ends it; FP32 vectors need a pass more when the
// recurrence residual has drifted from the true one.
template <typename T>
void b_pcg(BatchPCG &B, const double *b, double *x, int32_t *iters_h, double *res_h,
           grass_solve_stats_t *st) {
    grass_ctx_t ctx = B.ctx;
    grass_tree_t Tr = B.S->tree;
    const GraphData &g = Tr->g;
    const int64_t n = B.n, nc = B.ch.count, G = B.G;
    const int64_t *cb = B.ch.beg.p;
    const int32_t *cs = B.ch.seg.p;
    const int *act = B.act.p;
    std::vector<DBuf<T>> bufs(11);
    for (auto &bf : bufs) bf.alloc(n);
    BVecs<T> v{bufs[0].p, bufs[1].p, bufs[2].p, bufs[3].p, bufs[4].p, bufs[5].p,
               bufs[6].p, bufs[7].p, bufs[8].p, bufs[9].p, bufs[10].p};
    DBuf<double> r64;
    r64.alloc(n);
    BMat<T> A, MS;
    if constexpr (sizeof(T) == 8) {
        A = {g.adj_ptr.p, g.adj_col.p, g.adj_w64.p, g.D64.p};
        MS = {B.S->s_ptr.p, B.S->s_col.p, B.S->s_w64.p, g.D64.p};
    } else {
        A = {g.adj_ptr.p, g.adj_col.p, g.adj_w32.p, g.D32.p};
        MS = {B.S->s_ptr.p, B.S->s_col.p, B.S->s_w32.p, g.D32.p};
    }
    // x = 0, r = b, ||b||^2 per graph
    memset_d(ctx, x, 0, n * sizeof(double));
    copy_d(ctx, r64.p, b, n * sizeof(double));
    std::vector<int> need(G, 1);
    h2d(ctx, B.inpass.p, need.data(), G * sizeof(int));
    launch(ctx, k_b_dot2<double>, nc, kBT, 0, cb, cs, (const int *)B.inpass.p,
           (const double *)r64.p, (const double *)r64.p, (const double *)nullptr, B.part.p);
    B.sum(2, BS_BN);
    std::vector<double> bn(G), res(G), itp(G), itsum(G, 0.0), tolp(G);
    d2h(ctx, bn.data(), B.slot(BS_BN), G * sizeof(double));
    // first pass: the tolerance with some room for FP32 drift
    for (int64_t k = 0; k < G; ++k) {
        need[k] = bn[k] > 0.0 ? 1 : 0;
        tolp[k] = B.tol * (sizeof(T) == 4 ? 0.5 : 1.0);
    }

    auto iteration = [&]() {
        launch(ctx, k_b_matvec<T>, nc, kBT, 0, cb, cs, act, A, (const T *)v.P, v.Q, B.part.p);
        B.sum(1, BS_PQ);
        launch(ctx, k_bs_alpha, B.sgrid(), kBT, 0, G, (int)BS_RZ, (int)BS_PQ, (int)BS_ALPHA,
               B.sc.p, B.act.p, 1);
        launch(ctx, k_b_update<T>, nc, kBT, 0, cb, cs, act, (const double *)B.slot(BS_ALPHA), v.X,
               (const T *)v.P, v.R, (const T *)v.Q, v.Z, B.part.p);
        B.sum(1, BS_RR);
        GCK(cudaMemsetAsync(B.nact.p, 0, sizeof(int), ctx->stream));
        launch(ctx, k_bs_check, B.sgrid(), kBT, 0, G, B.maxit, B.sc.p, B.act.p, B.nact.p);
        b_precond<T>(B, v, MS);
        launch(ctx, k_b_dot2<T>, nc, kBT, 0, cb, cs, act, (const T *)v.R, (const T *)v.Z,
               (const T *)v.Zo, B.part.p);
        B.sum(2, BS_RZN);   // RZN, RZO
        launch(ctx, k_bs_beta, B.sgrid(), kBT, 0, G, BS_RZN, BS_RZO, BS_RZ, BS_BETA, B.sc.p, act);
        launch(ctx, k_b_pupd<T>, nc, kBT, 0, cb, cs, act, (const double *)B.slot(BS_BETA),
               (const T *)v.Z, v.P, v.Zo);
    };

    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool tried = false, captured = false;
    int64_t per = 0;
    constexpr int kMaxPasses = 8, kCheck = 4;
    int passes = 0;
    try {
        for (int pass = 0; pass < kMaxPasses; ++pass) {
            if (std::find(need.begin(), need.end(), 1) == need.end()) break;
            ++passes;
            h2d(ctx, B.inpass.p, need.data(), G * sizeof(int));
            h2d(ctx, B.slot(BS_TOL), tolp.data(), G * sizeof(double));
            // R = r, X = 0, ||R||^2, Z = M^{-1} R, P = Z, Zold = Z, rz = R.Z
            launch(ctx, k_b_pass<T>, nc, kBT, 0, cb, cs, (const int *)B.inpass.p,
                   (const double *)r64.p, v.R, v.X);
            launch(ctx, k_b_dot2<T>, nc, kBT, 0, cb, cs, (const int *)B.inpass.p, (const T *)v.R,
                   (const T *)v.R, (const T *)nullptr, B.part.p);
            B.sum(2, BS_BB);   // BB (and RR, which the init step overwrites)
            launch(ctx, k_bs_init, B.sgrid(), kBT, 0, G, B.sc.p, B.act.p, (const int *)B.inpass.p);
            launch(ctx, k_b_copy_act<T>, nc, kBT, 0, cb, cs, act, (const T *)v.R, v.Z, (T *)nullptr);
            b_precond<T>(B, v, MS);
            launch(ctx, k_b_copy_act<T>, nc, kBT, 0, cb, cs, act, (const T *)v.Z, v.P, (T *)nullptr);
            launch(ctx, k_b_copy_act<T>, nc, kBT, 0, cb, cs, act, (const T *)v.Z, v.Zo,
                   (T *)nullptr);
            launch(ctx, k_b_dot2<T>, nc, kBT, 0, cb, cs, act, (const T *)v.R, (const T *)v.Z,
                   (const T *)nullptr, B.part.p);
            B.sum(2, BS_RZN);
            launch(ctx, k_bs_beta, B.sgrid(), kBT, 0, G, BS_RZN, -1, BS_RZ, BS_BETA, B.sc.p, act);
            // iterations: the first one plain (it fills the launch-shape
            // caches), the rest replayed from a CUDA graph of one iteration
            iteration();
            int done = 1, nact = 0;
            d2h(ctx, &nact, B.nact.p, sizeof(int));
            if (!tried && nact > 0) {
                tried = true;
                const int64_t l0 = ctx->launches;
                // capture only on a capturable stream (not the legacy default
                // stream) and with kernel timing off
                cudaStreamCaptureStatus cs0 = cudaStreamCaptureStatusNone;
                const bool can = ctx->stream != nullptr && ctx->tfam == 0 &&
                                 cudaStreamIsCapturing(ctx->stream, &cs0) == cudaSuccess &&
                                 cs0 == cudaStreamCaptureStatusNone;
                if (can && cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) ==
                               cudaSuccess) {
                    bool ok = true;
                    try {
                        iteration();
                    } catch (...) {
                        ok = false;
                    }
                    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
                    captured = ok && e == cudaSuccess && graph &&
                               cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
                    if (!captured) cudaGetLastError();
                } else {
                    cudaGetLastError();
                }
                per = ctx->launches - l0;
                ctx->launches = l0;
            }
            while (nact > 0 && done < B.maxit) {
                for (int j = 0; j < kCheck && done < B.maxit; ++j, ++done) {
                    if (captured) {
                        GCK(cudaGraphLaunch(exec, ctx->stream));
                        ctx->launches += per;
                    } else {
                        iteration();
                    }
                }
                d2h(ctx, &nact, B.nact.p, sizeof(int));
            }
            // x += e in FP64, r = b - A x in FP64
            launch(ctx, k_b_accum<T>, nc, kBT, 0, cb, cs, (const int *)B.inpass.p, (const T *)v.X, x);
            launch(ctx, k_b_resid, nc, kBT, 0, cb, (const int32_t *)g.adj_ptr.p,
                   (const int32_t *)g.adj_col.p, (const double *)g.adj_w64.p,
                   (const double *)g.D64.p, (const double *)x, b, r64.p, B.part.p);
            B.sum(1, BS_RES);
            d2h(ctx, res.data(), B.slot(BS_RES), G * sizeof(double));
            d2h(ctx, itp.data(), B.slot(BS_IT), G * sizeof(double));
            for (int64_t k = 0; k < G; ++k) {
                if (need[k]) itsum[k] += itp[k];
                const double rel = bn[k] > 0.0 ? std::sqrt(res[k] / bn[k]) : 0.0;
                need[k] = rel > B.tol && itsum[k] < B.maxit ? 1 : 0;
                // next pass: reach half the tolerance from this residual
                tolp[k] = std::min(0.5, 0.5 * B.tol / std::max(rel, 1e-300));
            }
        }
    } catch (...) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        throw;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    int itmax = 0;
    double relmax = 0.0;
    for (int64_t k = 0; k < G; ++k) {
        double rel = bn[k] > 0.0 ? std::sqrt(res[k] / bn[k]) : 0.0;
        relmax = std::max(relmax, rel);
        itmax = std::max(itmax, (int)itsum[k]);
        if (iters_h) iters_h[k] = (int32_t)itsum[k];
        if (res_h) res_h[k] = rel;
    }
    st->iters = itmax;
    st->refinements = passes;
    st->inner_iters = (int64_t)itmax * std::max(B.inner, 0);
    st->rel_resid_fp64 = relmax;
    if (relmax > B.tol) fail(GRASS_ERR_NOT_CONVERGED, "a graph of the batch missed the tolerance");
}

}  // namespace
}  // namespace grass

using namespace grass;

#define BATCH_BEGIN(ctx)  \
    try {                 \
        GCK(cudaSetDevice((ctx)->device));
#define BATCH_END(ctx)                          \
    }                                           \
    catch (const Error &e) {                    \
        (ctx)->err = e.msg;                     \
        return e.st;                            \
    }                                           \
    catch (const std::bad_alloc &) {            \
        (ctx)->err = "host allocation failed";  \
        return GRASS_ERR_OOM;                   \
    }                                           \
    catch (...) {                               \
        (ctx)->err = "unexpected internal error"; \
        return GRASS_ERR_CUDA;                  \
    }                                           \
    return GRASS_OK;

static void need_b(bool ok, const char *msg) {
    if (!ok) fail(GRASS_ERR_INVALID, msg);
}

extern "C" grass_status grass_densify_batch(grass_ctx_t ctx, grass_tree_t T, const grass_params_t *P,
                                            const double *h0, const double *v0,
                                            grass_sparsifier_t *out, grass_sparsify_stats_t *stats,
                                            double *per_graph) {
    if (!ctx || !T || !P || !out) return GRASS_ERR_INVALID;
    BATCH_BEGIN(ctx)
    *out = nullptr;
    need_b(h0 && v0, "null h0 / v0");
    need_b(P->sigma2 > 0, "sigma2 must be > 0");
    need_b(r_supported(P->r), "r must be 1, 2, 4, 8, 16, 24 or 32");
    need_b(P->t >= 1, "t must be >= 1");
    need_b(P->max_rounds == 1, "the batched form runs one densification round (max_rounds = 1)");
    need_b(P->lmax_iters >= 0, "lmax_iters must be >= 0");
    need_b(P->max_add_per_round <= 0, "the batched form keeps every edge over the threshold (no cap)");
    need_b(P->embed_prec == GRASS_FP64 || P->embed_prec == GRASS_FP32, "bad embed_prec");
    const double t0 = now_ms();
    const GraphData &g = T->g;
    const int64_t n = g.n, G = g.nseg;
    const grass_prec prec = P->embed_prec;
    const size_t es = prec == GRASS_FP64 ? 8 : 4;
    grass_sparsify_stats_t st;
    std::memset(&st, 0, sizeof(st));
    clear_timeout(ctx);
    grass_sparsifier_t S = new_sparsifier(ctx, T);
    try {
        Chunks rows, edges;
        rows.build(ctx, g.seg_voff, kRowChunk);
        edges.build(ctx, g.seg_eoff, kEdgeChunk);
        DBuf<unsigned long long> bits;
        bits.alloc(G);
        DBuf<double> part, q;
        part.alloc(2 * std::max<int64_t>(edges.count, rows.count) + 2);
        q.alloc(2 * G);
        // lambda_min per graph (Sec. IV-C-2)
        const double ta = now_ms();
        launch(ctx, k_bits_init, cdiv(G, kBT), kBT, 0, G, bits.p, 0x7FF0000000000000ULL);
        launch(ctx, k_b_lmin, rows.count, kBT, 0, (const int64_t *)rows.beg.p,
               (const int32_t *)rows.seg.p, (const double *)g.degG.p, (const double *)S->degS.p,
               bits.p);
        std::vector<double> lmin(G), lmax(G), qq(2 * G), hmax(G), thr(G), theta(G);
        d2h(ctx, lmin.data(), bits.p, G * sizeof(double));
        // lambda_max per graph (Sec. IV-C-1): power steps with the forest
        // solve, then the per-graph Rayleigh quotient
        void *vv = ctx->scr<char>(SCR_LMAX_V, n * es);
        void *vy = ctx->scr<char>(SCR_LMAX_Y, n * es);
        if (P->lmax_iters > 0) {
            int slot = -1;
            power_steps(ctx, S, v0, 1, P->lmax_iters, prec, P->inner_tol, P->inner_maxit, vv, vy,
                        &slot);
            apply_pow2(ctx, prec, n, vv, maxslot(ctx, slot));
        } else {
            convert_block(ctx, prec, n, v0, vv);
        }
        if (prec == GRASS_FP64)
            launch(ctx, k_b_quad<double>, edges.count, kBT, 0, (const int64_t *)edges.beg.p,
                   (const int32_t *)g.eu.p, (const int32_t *)g.ev.p, (const double *)g.ew64.p,
                   (const uint8_t *)S->in_s.p, (const double *)vv, part.p);
        else
            launch(ctx, k_b_quad<float>, edges.count, kBT, 0, (const int64_t *)edges.beg.p,
                   (const int32_t *)g.eu.p, (const int32_t *)g.ev.p, (const double *)g.ew64.p,
                   (const uint8_t *)S->in_s.p, (const float *)vv, part.p);
        launch(ctx, k_b_sum, cdiv(G * 32, kBT), kBT, 0, G, 2, (const int32_t *)edges.first.p,
               (const double *)part.p, q.p);
        d2h(ctx, qq.data(), q.p, 2 * G * sizeof(double));
        check_timeout(ctx);
        int64_t active = 0;
        for (int64_t k = 0; k < G; ++k) {
            if (!(qq[G + k] > 0.0)) fail(GRASS_ERR_INVALID, "v^T L_S v is not positive for a graph");
            lmax[k] = qq[k] / qq[G + k];
            const bool similar = lmax[k] / lmin[k] <= P->sigma2;
            theta[k] = similar ? INFINITY : theta_sigma(P->sigma2, lmin[k], lmax[k], P->t);
            active += !similar;
        }
        const double tb = now_ms();
        st.ms_estimate = tb - ta;
        st.lmin_est[0] = *std::min_element(lmin.begin(), lmin.end());
        st.lmax_est[0] = *std::max_element(lmax.begin(), lmax.end());
        std::vector<int64_t> added(G, 0), moff_g(G, 0);
        if (active == 0) {
            st.stopped_similar = 1;
        } else {
            // embedding (Sec. III-F) over the whole batch, heat of every
            // off-forest edge, heat_max per graph
            void *H = ctx->scr<char>(SCR_H, n * P->r * es);
            void *Y = ctx->scr<char>(SCR_Y, n * P->r * es);
            int slot = 0;
            int64_t inner = power_steps(ctx, S, h0, P->r, P->t, prec, P->inner_tol, P->inner_maxit,
                                        H, Y, &slot);
            void *heat = ctx->scr<char>(SCR_HEAT, (S->m_off + 1) * es);
            heat_offs(ctx, P->r, prec, S, H, maxslot(ctx, slot), heat, maxslot(ctx, 2));
            const std::vector<int64_t> ooff = offtree_offsets(ctx, S);
            Chunks offc;
            offc.build(ctx, ooff, kEdgeChunk);
            launch(ctx, k_bits_init, cdiv(G, kBT), kBT, 0, G, bits.p, 0ULL);
            if (prec == GRASS_FP64)
                launch(ctx, k_b_hmax<double>, offc.count, kBT, 0, (const int64_t *)offc.beg.p,
                       (const int32_t *)offc.seg.p, (const double *)heat, bits.p);
            else
                launch(ctx, k_b_hmax<float>, offc.count, kBT, 0, (const int64_t *)offc.beg.p,
                       (const int32_t *)offc.seg.p, (const float *)heat, bits.p);
            d2h(ctx, hmax.data(), bits.p, G * sizeof(double));
            const double tc = now_ms();
            st.ms_embed = tc - tb;
            st.ms_embed_round[0] = tc - tb;
            // filter (Eq. heatratio_final) with each graph's own threshold
            for (int64_t k = 0; k < G; ++k) {
                thr[k] = std::isinf(theta[k]) ? INFINITY : theta[k] * hmax[k];
                moff_g[k] = ooff[k + 1] - ooff[k];
            }
            DBuf<double> thr_d;
            thr_d.alloc(G);
            h2d(ctx, thr_d.p, thr.data(), G * sizeof(double));
            const int64_t moff = S->m_off;
            int64_t *flag = ctx->scr<int64_t>(SCR_FILTER, moff + 1);
            int64_t *pos = ctx->scr<int64_t>(SCR_FILTER2, moff + 1);
            int64_t *acc = ctx->scr<int64_t>(SCR_PCG_E, moff + 1);
            int64_t na = 0;
            if (moff > 0) {
                if (prec == GRASS_FP64)
                    launch(ctx, k_b_flag<double>, offc.count, kBT, 0, (const int64_t *)offc.beg.p,
                           (const int32_t *)offc.seg.p, (const double *)heat,
                           (const double *)thr_d.p, flag);
                else
                    launch(ctx, k_b_flag<float>, offc.count, kBT, 0, (const int64_t *)offc.beg.p,
                           (const int32_t *)offc.seg.p, (const float *)heat,
                           (const double *)thr_d.p, flag);
                scan_i64(ctx, flag, pos, moff, &na);
                launch(ctx, k_b_scatter, cdiv(moff, kBT), kBT, 0, moff, (const int64_t *)flag,
                       (const int64_t *)pos, (const int32_t *)S->off_eid.p, acc);
                // accepted per graph: prefix counts at the graph boundaries
                std::vector<int64_t> pb(G + 1);
                for (int64_t k = 0; k <= G; ++k) {
                    if (ooff[k] >= moff) pb[k] = na;
                    else d2h(ctx, &pb[k], pos + ooff[k], sizeof(int64_t));
                }
                for (int64_t k = 0; k < G; ++k) added[k] = pb[k + 1] - pb[k];
            }
            const double td = now_ms();
            st.ms_filter = td - tc;
            st.rounds = 1;
            st.embedded_round[0] = moff;
            st.offtree_embedded = moff;
            st.added_round[0] = na;
            st.added = na;
            st.theta[0] = *std::min_element(theta.begin(), theta.end());
            st.heat_max[0] = *std::max_element(hmax.begin(), hmax.end());
            st.inner_iters = inner;
            if (na > 0) sparsifier_add(ctx, S, acc, na);
            ctx->sync();
            st.ms_update = now_ms() - td;
        }
        check_timeout(ctx);
        if (per_graph)
            for (int64_t k = 0; k < G; ++k) {
                double *o = per_graph + 6 * k;
                o[0] = lmin[k];
                o[1] = lmax[k];
                o[2] = theta[k];
                o[3] = hmax[k];
                o[4] = (double)added[k];
                o[5] = (double)moff_g[k];
            }
    } catch (...) {
        delete S;
        throw;
    }
    st.ms_total = now_ms() - t0;
    if (stats) *stats = st;
    *out = S;
    BATCH_END(ctx)
}

extern "C" grass_status grass_pcg_solve_batch(grass_ctx_t ctx, grass_sparsifier_t S, const double *b,
                                              double *x, double tol, int maxit, grass_prec prec,
                                              int inner_maxit, grass_solve_stats_t *stats,
                                              int32_t *iters, double *rel_resid) {
    if (!ctx || !S) return GRASS_ERR_INVALID;
    grass_solve_stats_t st;
    std::memset(&st, 0, sizeof(st));
    const double t0 = now_ms();
    try {
        GCK(cudaSetDevice(ctx->device));
        need_b(b && x, "null b / x");
        need_b(tol > 0 && maxit >= 1, "tol must be > 0, maxit >= 1");
        need_b(prec == GRASS_FP64 || prec == GRASS_FP32, "bad prec");
        need_b(inner_maxit >= 0, "inner_maxit must be >= 0");
        grass_tree_t Tr = S->tree;
        ensure_sdd(ctx, Tr);
        clear_timeout(ctx);
        BatchPCG B;
        B.ctx = ctx;
        B.S = S;
        B.prec = prec;
        B.n = Tr->g.n;
        B.G = Tr->g.nseg;
        B.ch.build(ctx, Tr->g.seg_voff, kRowChunk);
        B.part.alloc(2 * B.ch.count + 2);
        B.sc.alloc((int64_t)BS_N * B.G);
        B.act.alloc(B.G);
        B.inpass.alloc(B.G);
        B.nact.alloc(1);
        memset_d(ctx, B.sc.p, 0, (size_t)BS_N * B.G * sizeof(double));
        B.inner = inner_maxit;
        B.tol = tol;
        B.maxit = maxit;
        try {
            if (prec == GRASS_FP64) b_pcg<double>(B, b, x, iters, rel_resid, &st);
            else b_pcg<float>(B, b, x, iters, rel_resid, &st);
            check_timeout(ctx);
        } catch (...) {
            st.ms = now_ms() - t0;
            if (stats) *stats = st;
            throw;
        }
    } catch (const Error &e) {
        ctx->err = e.msg;
        return e.st;
    } catch (...) {
        ctx->err = "unexpected internal error";
        return GRASS_ERR_CUDA;
    }
    st.ms = now_ms() - t0;
    if (stats) *stats = st;
    return GRASS_OK;
}

// ---------------------------------------------------------------- autotuner
// Times the tree (forest) solve of `tree` for r columns under every launch
// shape below and keeps the fastest on the context: threads per block,
// blocks per SM, and the tail size (how many final rounds run in one block
// from shared memory).  The solve's results do not depend on the shape.

extern "C" grass_status grass_autotune(grass_ctx_t ctx, grass_tree_t T, int r, grass_prec prec,
                                       int64_t *best, double *best_ms) {
    if (!ctx || !T) return GRASS_ERR_INVALID;
    BATCH_BEGIN(ctx)
    need_b(r_supported(r), "r must be 1, 2, 4, 8, 16, 24 or 32");
    need_b(prec == GRASS_FP64 || prec == GRASS_FP32, "bad prec");
    const int64_t n = T->g.n;
    const size_t es = prec == GRASS_FP64 ? 8 : 4;
    clear_timeout(ctx);
    DBuf<char> Y;
    Y.alloc(n * r * es);
    memset_d(ctx, Y.p, 0, n * r * es);
    const int threads[] = {256, 512, 1024};
    const int bpsm[] = {1, 2, 4};
    const int64_t tails[] = {1024, 4096, 16384};
    const int keep_t = ctx->tree_threads, keep_b = ctx->tree_bpsm;
    const int64_t keep_tail = ctx->tree_tail_items;
    cudaEvent_t e0, e1;
    GCK(cudaEventCreate(&e0));
    GCK(cudaEventCreate(&e1));
    double bms = 1e300;
    int64_t b3[3] = {keep_t, keep_b, keep_tail};
    try {
        for (int th : threads)
            for (int bp : bpsm) {
                if (th * bp > 2048) continue;
                for (int64_t tl : tails) {
                    ctx->tree_threads = th;
                    ctx->tree_bpsm = bp;
                    ctx->tree_tail_items = tl;
                    tree_solve_inplace(ctx, T, T->lap, r, prec, Y.p, nullptr);   // warm
                    GCK(cudaEventRecord(e0, ctx->stream));
                    for (int k = 0; k < 3; ++k) tree_solve_inplace(ctx, T, T->lap, r, prec, Y.p, nullptr);
                    GCK(cudaEventRecord(e1, ctx->stream));
                    GCK(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    GCK(cudaEventElapsedTime(&ms, e0, e1));
                    if (ms / 3.0 < bms) {
                        bms = ms / 3.0;
                        b3[0] = th;
                        b3[1] = bp;
                        b3[2] = tl;
                    }
                }
            }
        check_timeout(ctx);
    } catch (...) {
        ctx->tree_threads = keep_t;
        ctx->tree_bpsm = keep_b;
        ctx->tree_tail_items = keep_tail;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tree_threads = (int)b3[0];
    ctx->tree_bpsm = (int)b3[1];
    ctx->tree_tail_items = b3[2];
    if (best) std::copy(b3, b3 + 3, best);
    if (best_ms) *best_ms = bms;
    BATCH_END(ctx)
}
