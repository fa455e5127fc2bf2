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
// grounded row rho is never eliminated; it is what remains at the end.  A
// batch of graphs (a spanning forest) has one such root per graph, and the
// rounds go on until only the roots remain.
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
__global__ void k_classify(int64_t n, const uint8_t *isroot, const int32_t *elim_round,
                           const int32_t *tptr, const int32_t *tocc, uint8_t *cls) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || elim_round[v] >= 0) return;
    int deg = 0;
    for (int32_t s = tptr[v]; s < tptr[v + 1]; ++s) deg += tocc[s] >= 0;
    uint8_t c = 0;
    if (!isroot[v]) c = deg == 1 ? 1 : (deg == 2 ? 2 : 0);
    cls[v] = c;
}

// Vertex id within its own graph: the compress priorities of a graph of a
// batch are those it has alone, so its elimination order (and rounding) does
// not depend on where it sits in the batch.
__device__ inline int32_t local_id(int32_t v, const int32_t *seg_of, const int64_t *voff) {
    return seg_of ? (int32_t)(v - voff[seg_of[v]]) : v;
}

__global__ void k_select(int64_t n, int round, const uint8_t *cls, const int32_t *tptr,
                         const int32_t *tocc, const int32_t *tsrc, const int32_t *seg_of,
                         const int64_t *voff, int32_t *elim_round, int32_t *n1, int32_t *n2,
                         int32_t *src1, int32_t *src2) {
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
    const int32_t lv = local_id((int32_t)v, seg_of, voff);
    if (ca == 2 && !prio_gt(lv, local_id(a, seg_of, voff), round)) return;
    if (cb == 2 && !prio_gt(lv, local_id(b, seg_of, voff), round)) return;
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

// ---------------------------------------------------------------- packed records

__global__ void k_pack_fwd(int64_t nr, const int32_t *rcv, const int32_t *beg, const int32_t *cv,
                           int4 *rec) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    int32_t b = beg[i], e = beg[i + 1];
    rec[i] = make_int4(rcv[i], cv[b], e - b >= 2 ? cv[b + 1] : -1, e - b >= 3 ? b + 2 : -1);
}

__global__ void k_pack_bwd(int64_t ne, const int32_t *elist, const int32_t *n1, const int32_t *n2,
                           int4 *rec) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ne) return;
    int32_t v = elist[p];
    rec[p] = make_int4(v, n1[v], n2[v], 0);
}

__global__ void k_tail_map(int64_t ne_tail, int64_t e0, const int32_t *elist, const int32_t *roots,
                           int64_t nroots, int64_t nt, int32_t *locmap, int32_t *tail_vid) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < ne_tail) {
        int32_t v = elist[e0 + p];
        locmap[v] = (int32_t)p;
        tail_vid[p] = v;
    } else if (p < ne_tail + nroots) {
        int32_t v = roots[p - ne_tail];
        locmap[v] = (int32_t)(nt - nroots + (p - ne_tail));
        tail_vid[nt - nroots + (p - ne_tail)] = v;
    }
}

__global__ void k_tail_fwd(int64_t cnt, const int4 *rec, const int32_t *locmap, int4 *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    int4 r = rec[i];
    out[i] = make_int4(locmap[r.x], locmap[r.y], r.z >= 0 ? locmap[r.z] : -1, r.w);
}

__global__ void k_tail_bwd(int64_t cnt, const int4 *rec, const int32_t *locmap, int4 *out) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= cnt) return;
    int4 r = rec[p];
    out[p] = make_int4(locmap[r.x], locmap[r.y], r.z >= 0 ? locmap[r.z] : -1, 0);
}

__global__ void k_tail_contrib(int64_t cnt, const int32_t *cv, const int32_t *locmap,
                               int32_t *out) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < cnt) out[c] = locmap[cv[c]];
}

// first contribution index of every round: beg[rcv_off[k]], k = 0..rounds
__global__ void k_round_contrib(int64_t cnt, const int64_t *rcv_off, const int32_t *beg,
                                int64_t *out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < cnt) out[k] = beg[rcv_off[k]];
}

// Vertices alive at the tail's first round: at most this many (local ids fit
// the shared-memory stage of the solve for small r).
constexpr int64_t kTailMax = 49152;

static void tree_pack(grass_ctx_t ctx, grass_tree_t T) {
    TreeSchedule &S = T->sched;
    const int64_t n = T->g.n, ne = n - T->nroots;
    S.fwd_rec.alloc(S.n_rcv);
    S.bwd_rec.alloc(ne);
    launch(ctx, k_pack_fwd, cdiv(S.n_rcv, kBlock), kBlock, 0, S.n_rcv,
           (const int32_t *)S.rcv_list.p, (const int32_t *)S.rcv_beg.p,
           (const int32_t *)S.contrib_v.p, S.fwd_rec.p);
    launch(ctx, k_pack_bwd, cdiv(ne, kBlock), kBlock, 0, ne, (const int32_t *)S.elim_list.p,
           (const int32_t *)S.n1.p, (const int32_t *)S.n2.p, S.bwd_rec.p);
    int k0 = 0;
    while (k0 < S.rounds && n - S.elim_off[k0] > kTailMax) ++k0;
    S.tail_k0 = k0;
    S.tail_n = n - S.elim_off[k0];
    const int64_t e0 = S.elim_off[k0], r0 = S.rcv_off[k0];
    DBuf<int32_t> locmap;
    locmap.alloc(n);
    S.tail_vid.alloc(S.tail_n);
    launch(ctx, k_tail_map, cdiv(ne - e0 + T->nroots, kBlock), kBlock, 0, ne - e0, e0,
           (const int32_t *)S.elim_list.p, (const int32_t *)T->roots.p, T->nroots, S.tail_n,
           locmap.p, S.tail_vid.p);
    S.fwd_loc.alloc(S.n_rcv - r0);
    S.bwd_loc.alloc(ne - e0);
    launch(ctx, k_tail_fwd, cdiv(S.n_rcv - r0, kBlock), kBlock, 0, S.n_rcv - r0,
           (const int4 *)S.fwd_rec.p + r0, (const int32_t *)locmap.p, S.fwd_loc.p);
    launch(ctx, k_tail_bwd, cdiv(ne - e0, kBlock), kBlock, 0, ne - e0,
           (const int4 *)S.bwd_rec.p + e0, (const int32_t *)locmap.p, S.bwd_loc.p);
    DBuf<int64_t> coff;
    coff.alloc(S.rounds + 1);
    launch(ctx, k_round_contrib, cdiv(S.rounds + 1, kBlock), kBlock, 0, (int64_t)S.rounds + 1,
           (const int64_t *)S.d_offs.p, (const int32_t *)S.rcv_beg.p, coff.p);
    S.contrib_off.assign(S.rounds + 1, 0);
    d2h(ctx, S.contrib_off.data(), coff.p, (S.rounds + 1) * sizeof(int64_t));
    const int64_t c0 = S.contrib_off[k0];
    S.tail_c0 = c0;
    S.contrib_loc.alloc(S.n_contrib - c0);
    launch(ctx, k_tail_contrib, cdiv(S.n_contrib - c0, kBlock), kBlock, 0, S.n_contrib - c0,
           (const int32_t *)S.contrib_v.p + c0, (const int32_t *)locmap.p, S.contrib_loc.p);
    ctx->sync();
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
    if (tslots != 2 * (n - T->nroots)) fail(GRASS_ERR_CUDA, "tree adjacency size mismatch");
    tocc.alloc(tslots);
    tsrc.alloc(tslots);
    launch(ctx, k_tfill, cdiv(n, kBlock), kBlock, 0, n, g.adj_ptr.p, g.adj_col.p, g.adj_eid.p,
           (const uint8_t *)T->in_tree.p, (const int64_t *)off.p, tptr.p, tocc.p, tsrc.p);
    // the scan form pays off while its FP64 tour arrays stay near the L2
    // size; larger trees keep the elimination rounds only
    if (n <= ctx->euler_max_n) euler_build(ctx, T, tptr.p, tocc.p, tsrc.p, tslots);
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
    while (alive > T->nroots) {
        if (round >= kMaxRounds) fail(GRASS_ERR_CUDA, "tree contraction did not finish");
        launch(ctx, k_classify, cdiv(n, kBlock), kBlock, 0, n, (const uint8_t *)T->isroot.p,
               (const int32_t *)elim_round.p, (const int32_t *)tptr.p, (const int32_t *)tocc.p,
               cls.p);
        launch(ctx, k_select, cdiv(n, kBlock), kBlock, 0, n, round, (const uint8_t *)cls.p,
               (const int32_t *)tptr.p, (const int32_t *)tocc.p, (const int32_t *)tsrc.p,
               g.nseg > 1 ? (const int32_t *)g.seg_of.p : nullptr,
               g.nseg > 1 ? (const int64_t *)g.seg_voff_d.p : nullptr, elim_round.p, S.n1.p,
               S.n2.p, S.src1.p, S.src2.p);
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
    tree_pack(ctx, T);
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

__global__ void k_nf_root(int64_t nroots, const int32_t *roots, const double *Dp, double *invd,
                          double *b1, double *b2, double *r64, float *r32) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nroots) return;
    const int32_t rho = roots[q];
    double d = Dp[rho];
    double iv = d > 0.0 ? 1.0 / d : 0.0;   // D = 0: grounded, x_rho = 0
    invd[rho] = iv;
    b1[rho] = 0.0;
    b2[rho] = 0.0;
    r64[q] = iv;
    r32[q] = (float)iv;
}

__global__ void k_to_f32(int64_t cnt, const double *a, float *b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) b[i] = (float)a[i];
}

__global__ void k_pack_fm(int64_t nr, const int32_t *beg, const double *cm, double2 *f64,
                          float2 *f32) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    int32_t b = beg[i], e = beg[i + 1];
    double m0 = cm[b], m1 = e - b >= 2 ? cm[b + 1] : 0.0;
    f64[i] = make_double2(m0, m1);
    f32[i] = make_float2((float)m0, (float)m1);
}

__global__ void k_pack_bc(int64_t ne, const int32_t *elist, const double *invd, const double *b1,
                          const double *b2, Dbl4 *c64, float4 *c32) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ne) return;
    int32_t v = elist[p];
    Dbl4 d{invd[v], b1[v], b2[v], 0.0};
    c64[p] = d;
    c32[p] = make_float4((float)d.x, (float)d.y, (float)d.z, 0.f);
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
    f.rinv64.alloc(T->nroots);
    f.rinv32.alloc(T->nroots);
    launch(ctx, k_nf_root, cdiv(T->nroots, kBlock), kBlock, 0, T->nroots,
           (const int32_t *)T->roots.p, (const double *)Dp.p, f.invd64.p, f.b1_64.p, f.b2_64.p,
           f.rinv64.p, f.rinv32.p);
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
    f.fm64.alloc(S.n_rcv);
    f.fm32.alloc(S.n_rcv);
    const int64_t ne = n - T->nroots;
    f.bc64.alloc(ne);
    f.bc32.alloc(ne);
    launch(ctx, k_pack_fm, cdiv(S.n_rcv, kBlock), kBlock, 0, S.n_rcv, (const int32_t *)S.rcv_beg.p,
           (const double *)f.cm64.p, f.fm64.p, f.fm32.p);
    launch(ctx, k_pack_bc, cdiv(ne, kBlock), kBlock, 0, ne, (const int32_t *)S.elim_list.p,
           (const double *)f.invd64.p, (const double *)f.b1_64.p, (const double *)f.b2_64.p,
           f.bc64.p, f.bc32.p);
    ctx->sync();
}

}  // namespace grass
