// tree.cu -- elimination schedule, numeric factorization and solves of the
// spanning-tree matrix L_T (+ D).
//
// Sec. III-H: a tree Laplacian factors in linear time.  The sequential
// textbook order eliminates leaves first and needs as many dependent steps
// as the tree is deep (tens of thousands on large meshes).  Here the tree is
// contracted in rounds instead: every round eliminates all current leaves
// (rake) and an independent set of degree-2 vertices (compress: the two
// neighbours get joined by the series edge w1 w2 / d).  Each round is a
// fixed set of independent eliminations, so the factor is the same
// Gaussian elimination in another order, with O(log n) rounds.  The
// grounded row rho is never eliminated; it is what remains at the end.
//
// Pivots are formed without subtraction: with Dp(v) the load collected from
// already-eliminated neighbours, d_v = Dp(v) + sum of v's current edge
// weights, and an elimination passes w * Dp(v) / d_v to each neighbour.
// For D = 0 every Dp stays exactly 0 and the final pivot of rho is 0: the
// solve is grounded there (x_rho = 0), the limit of the tiny diagonal on one
// row of Sec. III-F.
#include "common.cuh"

namespace grass {

__device__ inline uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ inline bool prio_gt(int32_t a, int32_t b, int round) {
    uint32_t ha = fmix32((uint32_t)a * 0x9E3779B1u + (uint32_t)round * 0x7F4A7C15u);
    uint32_t hb = fmix32((uint32_t)b * 0x9E3779B1u + (uint32_t)round * 0x7F4A7C15u);
    return ha != hb ? ha > hb : a > b;
}

// ---------------------------------------------------------------- tree adjacency

__global__ void k_tcount(int64_t n, const int32_t *adj_ptr, const int32_t *adj_eid,
                         const uint8_t *in_tree, int64_t *cnt) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t c = 0;
    for (int32_t j = adj_ptr[p]; j < adj_ptr[p + 1]; ++j) c += in_tree[adj_eid[j]];
    cnt[p] = c;
}

__global__ void k_tfill(int64_t n, const int32_t *adj_ptr, const int32_t *adj_col,
                        const int32_t *adj_eid, const uint8_t *in_tree, const int64_t *off,
                        int32_t *tptr, int32_t *tocc, int32_t *tsrc) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t k = off[p];
    tptr[p] = (int32_t)k;
    if (p == n - 1) tptr[n] = (int32_t)off[n];
    for (int32_t j = adj_ptr[p]; j < adj_ptr[p + 1]; ++j) {
        int32_t e = adj_eid[j];
        if (!in_tree[e]) continue;
        tocc[k] = adj_col[j];
        tsrc[k] = e;
        ++k;
    }
}

// ---------------------------------------------------------------- symbolic rounds

// cls: 0 stays, 1 leaf (rake), 2 degree two (compress candidate)
__global__ void k_classify(int64_t n, int32_t ground, const int32_t *elim_round,
                           const int32_t *tptr, const int32_t *tocc, uint8_t *cls) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || elim_round[v] >= 0) return;
    int deg = 0;
    for (int32_t s = tptr[v]; s < tptr[v + 1]; ++s) deg += tocc[s] >= 0;
    uint8_t c = 0;
    if (v != ground) c = deg == 1 ? 1 : (deg == 2 ? 2 : 0);
    cls[v] = c;
}

__global__ void k_select(int64_t n, int round, const uint8_t *cls, const int32_t *tptr,
                         const int32_t *tocc, const int32_t *tsrc, int32_t *elim_round,
                         int32_t *n1, int32_t *n2, int32_t *src1, int32_t *src2) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || elim_round[v] >= 0) return;
    uint8_t c = cls[v];
    if (c == 0) return;
    int32_t a = -1, b = -1, sa = 0, sb = 0;
    for (int32_t s = tptr[v]; s < tptr[v + 1]; ++s) {
        int32_t o = tocc[s];
        if (o < 0) continue;
        if (a < 0) {
            a = o;
            sa = tsrc[s];
        } else {
            b = o;
            sb = tsrc[s];
        }
    }
    if (c == 1) {
        elim_round[v] = round;
        n1[v] = a;
        src1[v] = sa;
        n2[v] = -1;
        src2[v] = 0;
        return;
    }
    // compress only between two survivors, and never next to another chosen
    // compress: v must beat every degree-2 neighbour on a per-round priority.
    uint8_t ca = cls[a], cb = cls[b];
    if (ca == 1 || cb == 1) return;
    if (ca == 2 && !prio_gt((int32_t)v, a, round)) return;
    if (cb == 2 && !prio_gt((int32_t)v, b, round)) return;
    elim_round[v] = round;
    n1[v] = a;
    src1[v] = sa;
    n2[v] = b;
    src2[v] = sb;
}

__global__ void k_count(int64_t n, int round, const int32_t *elim_round, const int32_t *tptr,
                        const int32_t *tocc, U64x2 *val) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t er = elim_round[v];
    U64x2 out{0ull, 0ull};
    if (er == round) {
        out.a = 1ull << 32;
    } else if (er < 0) {
        unsigned long long c = 0;
        for (int32_t s = tptr[v]; s < tptr[v + 1]; ++s) {
            int32_t o = tocc[s];
            if (o >= 0 && elim_round[o] == round) ++c;
        }
        if (c) {
            out.a = 1ull;
            out.b = c;
        }
    }
    val[v] = out;
}

__global__ void k_fill(int64_t n, int round, const int32_t *elim_round, const U64x2 *off,
                       int64_t ebase, int64_t rbase, int64_t cbase, const int32_t *n1,
                       const int32_t *n2, const int32_t *tptr, int32_t *tocc, int32_t *tsrc,
                       int32_t *elim_list, int32_t *rcv_list, int32_t *rcv_beg,
                       int32_t *contrib_v, uint8_t *contrib_side) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t er = elim_round[v];
    U64x2 o = off[v];
    if (er == round) {
        elim_list[ebase + (int64_t)(o.a >> 32)] = (int32_t)v;
        return;
    }
    if (er >= 0) return;
    // survivor: receiver if some neighbour went this round
    int64_t c = cbase + (int64_t)o.b;
    bool any = false;
    for (int32_t s = tptr[v]; s < tptr[v + 1]; ++s) {
        int32_t w = tocc[s];
        if (w < 0 || elim_round[w] != round) continue;
        any = true;
        bool side1 = n1[w] == (int32_t)v;
        contrib_v[c] = w;
        contrib_side[c] = side1 ? 0 : 1;
        ++c;
        int32_t other = n2[w] < 0 ? -1 : (side1 ? n2[w] : n1[w]);
        tocc[s] = other;                      // rake: slot empties; compress: series edge
        tsrc[s] = -(w + 1);
    }
    if (any) {
        int64_t ri = rbase + (int64_t)(o.a & 0xffffffffull);
        rcv_list[ri] = (int32_t)v;
        rcv_beg[ri] = (int32_t)(cbase + (int64_t)o.b);
    }
}

__global__ void k_set_i32(int64_t n, int32_t *a, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

void tree_schedule(grass_ctx_t ctx, grass_tree_t T) {
    const GraphData &g = T->g;
    const int64_t n = g.n;
    TreeSchedule &S = T->sched;
    DBuf<int32_t> tptr, tocc, tsrc, elim_round;
    DBuf<uint8_t> cls;
    DBuf<int64_t> cnt, off;
    DBuf<U64x2> val, voff;
    tptr.alloc(n + 1);
    cnt.alloc(n + 1);
    off.alloc(n + 1);
    launch(ctx, k_tcount, cdiv(n, kBlock), kBlock, 0, n, g.adj_ptr.p, g.adj_eid.p,
           (const uint8_t *)T->in_tree.p, cnt.p);
    int64_t tslots = 0;
    scan_i64(ctx, cnt.p, off.p, n, &tslots);
    if (tslots != 2 * (n - 1)) fail(GRASS_ERR_CUDA, "tree adjacency size mismatch");
    tocc.alloc(tslots);
    tsrc.alloc(tslots);
    launch(ctx, k_tfill, cdiv(n, kBlock), kBlock, 0, n, g.adj_ptr.p, g.adj_col.p, g.adj_eid.p,
           (const uint8_t *)T->in_tree.p, (const int64_t *)off.p, tptr.p, tocc.p, tsrc.p);
    elim_round.alloc(n);
    cls.alloc(n);
    val.alloc(n + 1);
    voff.alloc(n + 1);
    S.n1.alloc(n);
    S.n2.alloc(n);
    S.src1.alloc(n);
    S.src2.alloc(n);
    S.elim_list.alloc(n);
    S.rcv_list.alloc(2 * n);
    S.rcv_beg.alloc(2 * n + 1);
    S.contrib_v.alloc(2 * n);
    S.contrib_side.alloc(2 * n);
    launch(ctx, k_set_i32, cdiv(n, kBlock), kBlock, 0, n, elim_round.p, -1);
    launch(ctx, k_set_i32, cdiv(n, kBlock), kBlock, 0, n, S.n1.p, -1);
    launch(ctx, k_set_i32, cdiv(n, kBlock), kBlock, 0, n, S.n2.p, -1);
    memset_d(ctx, cls.p, 0, n);
    S.elim_off.assign(1, 0);
    S.rcv_off.assign(1, 0);
    int64_t alive = n, ebase = 0, rbase = 0, cbase = 0;
    int round = 0;
    while (alive > 1) {
        if (round > 4096) fail(GRASS_ERR_CUDA, "tree contraction did not finish");
        launch(ctx, k_classify, cdiv(n, kBlock), kBlock, 0, n, T->ground,
               (const int32_t *)elim_round.p, (const int32_t *)tptr.p, (const int32_t *)tocc.p,
               cls.p);
        launch(ctx, k_select, cdiv(n, kBlock), kBlock, 0, n, round, (const uint8_t *)cls.p,
               (const int32_t *)tptr.p, (const int32_t *)tocc.p, (const int32_t *)tsrc.p,
               elim_round.p, S.n1.p, S.n2.p, S.src1.p, S.src2.p);
        launch(ctx, k_count, cdiv(n, kBlock), kBlock, 0, n, round, (const int32_t *)elim_round.p,
               (const int32_t *)tptr.p, (const int32_t *)tocc.p, val.p);
        U64x2 tot{0, 0};
        scan_pair(ctx, val.p, voff.p, n, &tot);
        int64_t ne = (int64_t)(tot.a >> 32), nr = (int64_t)(tot.a & 0xffffffffull),
                nc = (int64_t)tot.b;
        if (ne == 0) fail(GRASS_ERR_CUDA, "tree contraction made no progress");
        launch(ctx, k_fill, cdiv(n, kBlock), kBlock, 0, n, round, (const int32_t *)elim_round.p,
               (const U64x2 *)voff.p, ebase, rbase, cbase, (const int32_t *)S.n1.p,
               (const int32_t *)S.n2.p, (const int32_t *)tptr.p, tocc.p, tsrc.p, S.elim_list.p,
               S.rcv_list.p, S.rcv_beg.p, S.contrib_v.p, S.contrib_side.p);
        ebase += ne;
        rbase += nr;
        cbase += nc;
        alive -= ne;
        S.elim_off.push_back(ebase);
        S.rcv_off.push_back(rbase);
        ++round;
    }
    S.rounds = round;
    S.n_rcv = rbase;
    S.n_contrib = cbase;
    int32_t sentinel = (int32_t)cbase;
    h2d(ctx, S.rcv_beg.p + rbase, &sentinel, sizeof(int32_t));
    std::vector<int64_t> h(2 * (S.rounds + 1));
    for (int k = 0; k <= S.rounds; ++k) {
        h[k] = S.rcv_off[k];
        h[S.rounds + 1 + k] = S.elim_off[k];
    }
    S.d_offs.alloc(h.size());
    h2d(ctx, S.d_offs.p, h.data(), h.size() * sizeof(int64_t));
}

// ---------------------------------------------------------------- numeric factorization

__device__ inline double src_weight(int32_t src, const double *ew, const double *fill) {
    return src >= 0 ? ew[src] : fill[-src - 1];
}

__global__ void k_nf_elim(int64_t cnt, const int32_t *elist, const int32_t *n2, const int32_t *src1,
                          const int32_t *src2, const double *ew, const double *Dp, double *fill,
                          double *invd, double *b1, double *b2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    int32_t v = elist[i];
    double w1 = src_weight(src1[v], ew, fill);
    double w2 = n2[v] >= 0 ? src_weight(src2[v], ew, fill) : 0.0;
    double d = Dp[v] + w1 + w2;
    invd[v] = 1.0 / d;
    b1[v] = w1 / d;
    b2[v] = w2 / d;
    fill[v] = n2[v] >= 0 ? w1 * w2 / d : 0.0;
}

__global__ void k_nf_rcv(int64_t cnt, const int32_t *rlist, const int32_t *beg,
                         const int32_t *cv, const uint8_t *side, const double *b1,
                         const double *b2, double *Dp) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    int32_t u = rlist[i];
    double s = Dp[u];
    for (int32_t k = beg[i]; k < beg[i + 1]; ++k) {
        int32_t v = cv[k];
        s += Dp[v] * (side[k] ? b2[v] : b1[v]);
    }
    Dp[u] = s;
}

__global__ void k_nf_cm(int64_t cnt, const int32_t *cv, const uint8_t *side, const double *b1,
                        const double *b2, double *cm) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    int32_t v = cv[k];
    cm[k] = side[k] ? b2[v] : b1[v];
}

__global__ void k_nf_root(int32_t rho, const double *Dp, double *invd, double *b1, double *b2,
                          double *out) {
    double d = Dp[rho];
    double iv = d > 0.0 ? 1.0 / d : 0.0;   // D = 0: grounded, x_rho = 0
    invd[rho] = iv;
    b1[rho] = 0.0;
    b2[rho] = 0.0;
    *out = iv;
}

__global__ void k_to_f32(int64_t cnt, const double *a, float *b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) b[i] = (float)a[i];
}

void tree_factor(grass_ctx_t ctx, grass_tree_t T, bool with_D, TreeFactor &f) {
    const GraphData &g = T->g;
    const TreeSchedule &S = T->sched;
    const int64_t n = g.n;
    f.invd64.alloc(n);
    f.b1_64.alloc(n);
    f.b2_64.alloc(n);
    f.fill64.alloc(n);
    f.cm64.alloc(S.n_contrib + 1);
    DBuf<double> Dp;
    Dp.alloc(n);
    if (with_D) copy_d(ctx, Dp.p, g.D64.p, n * sizeof(double));
    else memset_d(ctx, Dp.p, 0, n * sizeof(double));
    for (int k = 0; k < S.rounds; ++k) {
        int64_t e0 = S.elim_off[k], e1 = S.elim_off[k + 1];
        launch(ctx, k_nf_elim, cdiv(e1 - e0, kBlock), kBlock, 0, e1 - e0,
               (const int32_t *)S.elim_list.p + e0, (const int32_t *)S.n2.p,
               (const int32_t *)S.src1.p, (const int32_t *)S.src2.p, (const double *)g.ew64.p,
               (const double *)Dp.p, f.fill64.p, f.invd64.p, f.b1_64.p, f.b2_64.p);
        if (with_D) {
            int64_t r0 = S.rcv_off[k], r1 = S.rcv_off[k + 1];
            launch(ctx, k_nf_rcv, cdiv(r1 - r0, kBlock), kBlock, 0, r1 - r0,
                   (const int32_t *)S.rcv_list.p + r0, (const int32_t *)S.rcv_beg.p + r0,
                   (const int32_t *)S.contrib_v.p, (const uint8_t *)S.contrib_side.p,
                   (const double *)f.b1_64.p, (const double *)f.b2_64.p, Dp.p);
        }
    }
    double *dout = ctx->scal.p + DS_RED;
    launch(ctx, k_nf_root, 1, 1, 0, T->ground, (const double *)Dp.p, f.invd64.p, f.b1_64.p,
           f.b2_64.p, dout);
    launch(ctx, k_nf_cm, cdiv(S.n_contrib, kBlock), kBlock, 0, S.n_contrib,
           (const int32_t *)S.contrib_v.p, (const uint8_t *)S.contrib_side.p,
           (const double *)f.b1_64.p, (const double *)f.b2_64.p, f.cm64.p);
    f.invd32.alloc(n);
    f.b1_32.alloc(n);
    f.b2_32.alloc(n);
    f.cm32.alloc(S.n_contrib + 1);
    launch(ctx, k_to_f32, cdiv(n, kBlock), kBlock, 0, n, (const double *)f.invd64.p, f.invd32.p);
    launch(ctx, k_to_f32, cdiv(n, kBlock), kBlock, 0, n, (const double *)f.b1_64.p, f.b1_32.p);
    launch(ctx, k_to_f32, cdiv(n, kBlock), kBlock, 0, n, (const double *)f.b2_64.p, f.b2_32.p);
    launch(ctx, k_to_f32, cdiv(S.n_contrib, kBlock), kBlock, 0, S.n_contrib,
           (const double *)f.cm64.p, f.cm32.p);
    d2h(ctx, &f.root_invd, dout, sizeof(double));
}

// ---------------------------------------------------------------- solves

__device__ inline void atomic_max_abs(unsigned long long *maxbits, double v) {
    // warp max first, one atomic per warp; |v| >= 0 orders like its bits
    v = fabs(v);
    for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, d));
    if ((threadIdx.x & 31) == 0 && v > 0.0)
        atomicMax(maxbits, (unsigned long long)__double_as_longlong(v));
}

template <typename T, int R>
__device__ inline void fwd_item(int64_t i, int c, const int32_t *rcv, const int32_t *beg,
                                const int32_t *cv, const T *cm, T *Y) {
    constexpr int EPT = Lay<R>::EPT;
    int32_t u = rcv[i];
    T *yu = Y + (int64_t)u * R + c * EPT;
    T acc[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) acc[e] = yu[e];
    int32_t k1 = beg[i + 1];
    for (int32_t k = beg[i]; k < k1; ++k) {
        const T *yv = Y + (int64_t)cv[k] * R + c * EPT;
        T mlt = cm[k];
#pragma unroll
        for (int e = 0; e < EPT; ++e) acc[e] += mlt * yv[e];
    }
#pragma unroll
    for (int e = 0; e < EPT; ++e) yu[e] = acc[e];
}

template <typename T, int R>
__device__ inline double bwd_item(int32_t v, int c, const int32_t *n1, const int32_t *n2,
                                  const T *invd, const T *b1, const T *b2, T *Y) {
    constexpr int EPT = Lay<R>::EPT;
    T *yv = Y + (int64_t)v * R + c * EPT;
    int32_t a = n1[v], b = n2[v];
    T id = invd[v], c1 = b1[v];
    const T *xa = Y + (int64_t)a * R + c * EPT;
    T x[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) x[e] = id * yv[e] + c1 * xa[e];
    if (b >= 0) {
        T c2 = b2[v];
        const T *xb = Y + (int64_t)b * R + c * EPT;
#pragma unroll
        for (int e = 0; e < EPT; ++e) x[e] += c2 * xb[e];
    }
    double mx = 0.0;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        yv[e] = x[e];
        mx = fmax(mx, fabs((double)x[e]));
    }
    return mx;
}

template <typename T, int R>
__global__ void k_fwd_round(int64_t cnt, const int32_t *rcv, const int32_t *beg, const int32_t *cv,
                            const T *cm, T *Y) {
    constexpr int TPR = Lay<R>::TPR;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = t / TPR;
    if (i >= cnt) return;
    fwd_item<T, R>(i, (int)(t % TPR), rcv, beg, cv, cm, Y);
}

template <typename T, int R>
__global__ void k_bwd_round(int64_t cnt, const int32_t *elist, const int32_t *n1,
                            const int32_t *n2, const T *invd, const T *b1, const T *b2, T *Y,
                            unsigned long long *maxbits) {
    constexpr int TPR = Lay<R>::TPR;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = t / TPR;
    double mx = 0.0;
    if (i < cnt) mx = bwd_item<T, R>(elist[i], (int)(t % TPR), n1, n2, invd, b1, b2, Y);
    if (maxbits) atomic_max_abs(maxbits, mx);
}

// The last rounds are small: one block runs them all, forward, the root and
// backward, with block barriers between rounds instead of kernel launches.
template <typename T, int R>
__global__ void k_tail(int k0, int rounds, const int64_t *rcv_off, const int64_t *elim_off,
                       const int32_t *rcv, const int32_t *beg, const int32_t *cv, const T *cm,
                       const int32_t *elist, const int32_t *n1, const int32_t *n2, const T *invd,
                       const T *b1, const T *b2, int32_t rho, T *Y, unsigned long long *maxbits) {
    constexpr int TPR = Lay<R>::TPR, EPT = Lay<R>::EPT;
    const int items_per_pass = blockDim.x / TPR;
    const int c = threadIdx.x % TPR;
    const int slot = threadIdx.x / TPR;
    for (int k = k0; k < rounds; ++k) {
        for (int64_t i = rcv_off[k] + slot; i < rcv_off[k + 1]; i += items_per_pass)
            fwd_item<T, R>(i, c, rcv, beg, cv, cm, Y);
        __syncthreads();
    }
    double mx = 0.0;
    if (slot == 0) {
        T *yr = Y + (int64_t)rho * R + c * EPT;
        T id = invd[rho];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            yr[e] = id * yr[e];
            mx = fmax(mx, fabs((double)yr[e]));
        }
    }
    __syncthreads();
    for (int k = rounds - 1; k >= k0; --k) {
        for (int64_t i = elim_off[k] + slot; i < elim_off[k + 1]; i += items_per_pass)
            mx = fmax(mx, bwd_item<T, R>(elist[i], c, n1, n2, invd, b1, b2, Y));
        __syncthreads();
    }
    if (maxbits) atomic_max_abs(maxbits, mx);
}

struct SolveArgs {
    grass_ctx_t ctx;
    grass_tree_t T;
    const TreeFactor *f;
    void *Y;
    unsigned long long *maxbits;
    grass_prec prec;
};

// Rounds at or after the tail start run inside one block.
static int tail_start(const TreeSchedule &S) {
    const int64_t kTailItems = 4096;
    int k0 = S.rounds;
    int64_t items = 0;
    while (k0 > 0) {
        int k = k0 - 1;
        int64_t add = (S.rcv_off[k + 1] - S.rcv_off[k]) + (S.elim_off[k + 1] - S.elim_off[k]);
        if (items + add > kTailItems) break;
        items += add;
        k0 = k;
    }
    return k0;
}

// One cooperative launch per solve: the big rounds are separated by grid
// barriers instead of kernel boundaries, the small last rounds run in
// block 0 alone (block barriers), then the big rounds again backwards.
constexpr int kPersistThreads = 256;

template <typename T, int R>
__global__ void __launch_bounds__(kPersistThreads)
    k_tree_persist(int rounds, int k0, const int64_t *rcv_off, const int64_t *elim_off,
                   const int32_t *rcv, const int32_t *beg, const int32_t *cv, const T *cm,
                   const int32_t *elist, const int32_t *n1, const int32_t *n2, const T *invd,
                   const T *b1, const T *b2, int32_t rho, T *Y, unsigned long long *maxbits,
                   unsigned int *bar, long long budget, int *err) {
    constexpr int TPR = Lay<R>::TPR, EPT = Lay<R>::EPT;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = (int)(gt % TPR);
    const int64_t slot = gt / TPR;
    const int64_t nslots = (int64_t)gridDim.x * blockDim.x / TPR;
    for (int k = 0; k < k0; ++k) {
        const int64_t e = rcv_off[k + 1];
        for (int64_t i = rcv_off[k] + slot; i < e; i += nslots)
            fwd_item<T, R>(i, c, rcv, beg, cv, cm, Y);
        if (!grid_sync(bar, budget, err)) return;
    }
    double mx = 0.0;
    if (blockIdx.x == 0) {
        const int bslot = threadIdx.x / TPR, bslots = blockDim.x / TPR;
        for (int k = k0; k < rounds; ++k) {
            for (int64_t i = rcv_off[k] + bslot; i < rcv_off[k + 1]; i += bslots)
                fwd_item<T, R>(i, c, rcv, beg, cv, cm, Y);
            __syncthreads();
        }
        if (bslot == 0) {
            T *yr = Y + (int64_t)rho * R + c * EPT;
            T id = invd[rho];
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                yr[e] = id * yr[e];
                mx = fmax(mx, fabs((double)yr[e]));
            }
        }
        __syncthreads();
        for (int k = rounds - 1; k >= k0; --k) {
            for (int64_t i = elim_off[k] + bslot; i < elim_off[k + 1]; i += bslots)
                mx = fmax(mx, bwd_item<T, R>(elist[i], c, n1, n2, invd, b1, b2, Y));
            __syncthreads();
        }
    }
    if (k0 > 0 && !grid_sync(bar, budget, err)) return;
    for (int k = k0 - 1; k >= 0; --k) {
        const int64_t e = elim_off[k + 1];
        for (int64_t i = elim_off[k] + slot; i < e; i += nslots)
            mx = fmax(mx, bwd_item<T, R>(elist[i], c, n1, n2, invd, b1, b2, Y));
        if (k > 0 && !grid_sync(bar, budget, err)) return;
    }
    if (maxbits) block_atomic_max(maxbits, mx);
}

template <typename T, int R>
static void solve_persistent(const SolveArgs &a, const T *invd, const T *b1, const T *b2,
                             const T *cm) {
    grass_ctx_t ctx = a.ctx;
    const TreeSchedule &S = a.T->sched;
    static int blocks_per_sm = -1;   // per instantiation
    if (blocks_per_sm < 0) {
        int nb = 0;
        GCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tree_persist<T, R>,
                                                          kPersistThreads, 0));
        blocks_per_sm = nb;
    }
    if (blocks_per_sm < 1) fail(GRASS_ERR_CUDA, "persistent tree solve does not fit on an SM");
    int grid = ctx->num_sms * std::min(blocks_per_sm, 4);
    int rounds = S.rounds, k0 = tail_start(S);
    const int64_t *rcv_off = S.d_offs.p, *elim_off = S.d_offs.p + (S.rounds + 1);
    const int32_t *rcv = S.rcv_list.p, *beg = S.rcv_beg.p, *cv = S.contrib_v.p;
    const int32_t *elist = S.elim_list.p, *n1 = S.n1.p, *n2 = S.n2.p;
    int32_t rho = a.T->ground;
    T *Y = (T *)a.Y;
    unsigned long long *maxbits = a.maxbits;
    unsigned int *bar = ctx->gbar.p;
    long long budget = ctx->wait_budget;
    int *err = ctx->flags.p + 3;
    GCK(cudaMemsetAsync(bar, 0, sizeof(unsigned int), ctx->stream));
    void *args[] = {&rounds, &k0, &rcv_off, &elim_off, &rcv, &beg, &cv, &cm, &elist, &n1, &n2,
                    &invd, &b1, &b2, &rho, &Y, &maxbits, &bar, &budget, &err};
    GCK(cudaLaunchCooperativeKernel((const void *)k_tree_persist<T, R>, dim3(grid),
                                    dim3(kPersistThreads), args, 0, ctx->stream));
    ctx->launches++;
}

template <typename T, int R>
static void solve_T(const SolveArgs &a, const T *invd, const T *b1, const T *b2, const T *cm) {
    constexpr int TPR = Lay<R>::TPR;
    grass_ctx_t ctx = a.ctx;
    const TreeSchedule &S = a.T->sched;
    T *Y = (T *)a.Y;
    if (ctx->num_sms > 0) {
        solve_persistent<T, R>(a, invd, b1, b2, cm);
        return;
    }
    const int k0 = tail_start(S);
    for (int k = 0; k < k0; ++k) {
        int64_t r0 = S.rcv_off[k], cnt = S.rcv_off[k + 1] - r0;
        launch(ctx, k_fwd_round<T, R>, cdiv(cnt * TPR, kBlock), kBlock, 0, cnt,
               (const int32_t *)S.rcv_list.p + r0, (const int32_t *)S.rcv_beg.p + r0,
               (const int32_t *)S.contrib_v.p, cm, Y);
    }
    const int64_t *offs = S.d_offs.p;
    launch(ctx, k_tail<T, R>, 1, 1024, 0, k0, S.rounds, (const int64_t *)offs,
           (const int64_t *)offs + (S.rounds + 1), (const int32_t *)S.rcv_list.p,
           (const int32_t *)S.rcv_beg.p, (const int32_t *)S.contrib_v.p, cm,
           (const int32_t *)S.elim_list.p, (const int32_t *)S.n1.p, (const int32_t *)S.n2.p,
           invd, b1, b2, a.T->ground, Y, a.maxbits);
    for (int k = k0 - 1; k >= 0; --k) {
        int64_t e0 = S.elim_off[k], cnt = S.elim_off[k + 1] - e0;
        launch(ctx, k_bwd_round<T, R>, cdiv(cnt * TPR, kBlock), kBlock, 0, cnt,
               (const int32_t *)S.elim_list.p + e0, (const int32_t *)S.n1.p,
               (const int32_t *)S.n2.p, invd, b1, b2, Y, a.maxbits);
    }
}

template <int R>
static void solve_R(const SolveArgs &a) {
    const TreeFactor &f = *a.f;
    if (a.prec == GRASS_FP64)
        solve_T<double, R>(a, f.invd64.p, f.b1_64.p, f.b2_64.p, f.cm64.p);
    else
        solve_T<float, R>(a, f.invd32.p, f.b1_32.p, f.b2_32.p, f.cm32.p);
}

void tree_solve_inplace(grass_ctx_t ctx, grass_tree_t T, const TreeFactor &f, int r,
                        grass_prec prec, void *Y, unsigned long long *maxbits) {
    SolveArgs a{ctx, T, &f, Y, maxbits, prec};
    const TreeSchedule &S = T->sched;
    const double s = prec == GRASS_FP64 ? 8.0 : 4.0, n = (double)T->g.n;
    const double bytes = 4.0 * n * r * s + S.n_contrib * (4.0 + s) + S.n_rcv * 8.0 + n * (12.0 + 3.0 * s);
    bool timed = ctx->t_begin(GRASS_KF_TREE, bytes);
    GRASS_DISPATCH_R(r, solve_R, a);
    ctx->t_end(timed);
}

}  // namespace grass
