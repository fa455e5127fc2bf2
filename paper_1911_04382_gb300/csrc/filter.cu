// filter.cu -- sparsifier bookkeeping (edge mask, off-sparsifier edge list,
// sparsifier adjacency, weighted degrees), the lambda_min estimate and the
// Joule-heat threshold filter with optional radix-select cap.
#include "common.cuh"

namespace grass {

// ---------------------------------------------------------------- sparsifier state

__global__ void k_off_flag(int64_t m, const uint8_t *in_s, int64_t *flag) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) flag[e] = in_s[e] ? 0 : 1;
}

__global__ void k_off_fill(int64_t m, const uint8_t *in_s, const int64_t *pos, const int32_t *eu,
                           const int32_t *ev, const double *ew, int32_t *ou, int32_t *ov,
                           int32_t *oe, double *ow, float *ow32) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m || in_s[e]) return;
    int64_t k = pos[e];
    ou[k] = eu[e];
    ov[k] = ev[e];
    oe[k] = (int32_t)e;
    ow[k] = ew[e];
    ow32[k] = (float)ew[e];
}

__global__ void k_s_count(int64_t n, const int32_t *adj_ptr, const int32_t *adj_eid,
                          const double *adj_w, const uint8_t *in_s, int64_t *cnt, double *degS) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t c = 0;
    double d = 0.0;
    for (int32_t j = adj_ptr[p]; j < adj_ptr[p + 1]; ++j)
        if (in_s[adj_eid[j]]) {
            ++c;
            d += adj_w[j];
        }
    cnt[p] = c;
    degS[p] = d;
}

__global__ void k_s_fill(int64_t n, const int32_t *adj_ptr, const int32_t *adj_col,
                         const int32_t *adj_eid, const double *adj_w, const uint8_t *in_s,
                         const int64_t *off, int32_t *s_ptr, int32_t *s_col, double *s_w,
                         float *s_w32) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t k = off[p];
    s_ptr[p] = (int32_t)k;
    if (p == n - 1) s_ptr[n] = (int32_t)off[n];
    for (int32_t j = adj_ptr[p]; j < adj_ptr[p + 1]; ++j)
        if (in_s[adj_eid[j]]) {
            s_col[k] = adj_col[j];
            s_w[k] = adj_w[j];
            s_w32[k] = (float)adj_w[j];
            ++k;
        }
}

void sparsifier_rebuild(grass_ctx_t ctx, grass_sparsifier_t S) {
    const GraphData &g = S->tree->g;
    const int64_t n = g.n, m = g.m;
    int64_t *flag = ctx->scr<int64_t>(SCR_TMP0, m + 1);
    int64_t *pos = ctx->scr<int64_t>(SCR_TMP1, m + 1);
    launch(ctx, k_off_flag, cdiv(m, kBlock), kBlock, 0, m, (const uint8_t *)S->in_s.p, flag);
    int64_t moff = 0;
    scan_i64(ctx, flag, pos, m, &moff);
    S->off_u.reserve(moff);
    S->off_v.reserve(moff);
    S->off_eid.reserve(moff);
    S->off_w64.reserve(moff);
    S->off_w32.reserve(moff);
    launch(ctx, k_off_fill, cdiv(m, kBlock), kBlock, 0, m, (const uint8_t *)S->in_s.p,
           (const int64_t *)pos, g.eu.p, g.ev.p, g.ew64.p, S->off_u.p, S->off_v.p, S->off_eid.p,
           S->off_w64.p, S->off_w32.p);
    S->m_off = moff;
    S->n_edges = m - moff;
    S->is_tree = S->n_edges == n - S->tree->nroots;
    S->degS.reserve(n);
    int64_t *cnt = ctx->scr<int64_t>(SCR_TMP2, n + 1);
    int64_t *off = ctx->scr<int64_t>(SCR_TMP3, n + 1);
    launch(ctx, k_s_count, cdiv(n, kBlock), kBlock, 0, n, g.adj_ptr.p, g.adj_eid.p, g.adj_w64.p,
           (const uint8_t *)S->in_s.p, cnt, S->degS.p);
    if (!S->is_tree) {
        int64_t ns = 0;
        scan_i64(ctx, cnt, off, n, &ns);
        S->s_nnz = ns;
        S->s_ptr.reserve(n + 1);
        S->s_col.reserve(ns);
        S->s_w64.reserve(ns);
        S->s_w32.reserve(ns);
        launch(ctx, k_s_fill, cdiv(n, kBlock), kBlock, 0, n, g.adj_ptr.p, g.adj_col.p, g.adj_eid.p,
               g.adj_w64.p, (const uint8_t *)S->in_s.p, (const int64_t *)off, S->s_ptr.p,
               S->s_col.p, S->s_w64.p, S->s_w32.p);
        heavy_rows(ctx, n, ns, S->s_ptr.p, S->s_heavy);
    } else {
        S->s_heavy.count = 0;
    }
    S->pre_ok = false;
    S->amg[0].reset();
    S->amg[1].reset();
}

__global__ void k_mark(int64_t cnt, const int64_t *eids, int64_t m, uint8_t *in_s, int *flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    int64_t e = eids[i];
    if (e < 0 || e >= m) {
        atomicOr(flags, 1);
        return;
    }
    in_s[e] = 1;
}

void sparsifier_add(grass_ctx_t ctx, grass_sparsifier_t S, const int64_t *eids, int64_t count) {
    if (count < 0) fail(GRASS_ERR_INVALID, "negative edge count");
    if (count == 0) return;
    memset_d(ctx, ctx->flags.p, 0, sizeof(int));
    launch(ctx, k_mark, cdiv(count, kBlock), kBlock, 0, count, eids, S->tree->g.m, S->in_s.p,
           ctx->flags.p);
    int f = 0;
    d2h(ctx, &f, ctx->flags.p, sizeof(int));
    sparsifier_rebuild(ctx, S);
    if (f) fail(GRASS_ERR_INVALID, "edge id out of range (valid ids were still added)");
}

// ---------------------------------------------------------------- lambda_min (Eq. courant-fischer-3)

__global__ void k_lmin(int64_t n, const double *degG, const double *degS, unsigned long long *out) {
    double mn = 1.0 / 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        mn = fmin(mn, degG[p] / degS[p]);
    for (int d = 16; d > 0; d >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, d));
    if ((threadIdx.x & 31) == 0) atomicMin(out, (unsigned long long)__double_as_longlong(mn));
}

void lambda_min(grass_ctx_t ctx, grass_sparsifier_t S, double *out_host) {
    const GraphData &g = S->tree->g;
    unsigned long long *o = (unsigned long long *)(ctx->scal.p + DS_MAX + 8);
    unsigned long long init = 0x7FF0000000000000ULL;   // +inf
    GCK(cudaMemcpyAsync(o, &init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream));
    int64_t grid = std::min<int64_t>(kRedBlocks, cdiv(g.n, kBlock));
    launch(ctx, k_lmin, grid, kBlock, 0, g.n, (const double *)g.degG.p,
           (const double *)S->degS.p, o);
    d2h(ctx, out_host, o, sizeof(double));
}

// ---------------------------------------------------------------- filter

template <typename T>
__global__ void k_thr_flag(int64_t moff, const T *heat, double thr, int64_t *flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < moff) flag[i] = (double)heat[i] >= thr ? 1 : 0;
}

__global__ void k_scatter_ids(int64_t moff, const int64_t *flag, const int64_t *pos,
                              const int32_t *off_eid, int64_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < moff && flag[i]) out[pos[i]] = off_eid[i];
}

template <typename T>
__device__ inline unsigned long long key_of(T h);
template <>
__device__ inline unsigned long long key_of<float>(float h) { return (unsigned long long)__float_as_uint(h); }
template <>
__device__ inline unsigned long long key_of<double>(double h) { return (unsigned long long)__double_as_longlong(h); }

// histogram of one 8-bit digit over candidates (heat >= thr) whose key
// matches the prefix found so far
template <typename T>
__global__ void k_radix_hist(int64_t moff, const T *heat, double thr, unsigned long long prefix,
                             unsigned long long mask, int shift, unsigned int *hist) {
    __shared__ unsigned int h[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < moff;
         i += (int64_t)gridDim.x * blockDim.x) {
        T x = heat[i];
        if (!((double)x >= thr)) continue;
        unsigned long long k = key_of<T>(x);
        if ((k & mask) != prefix) continue;
        atomicAdd(&h[(k >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

template <typename T>
__global__ void k_sel_flags(int64_t moff, const T *heat, double thr, unsigned long long kstar,
                            int64_t *gt, int64_t *eq) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= moff) return;
    T x = heat[i];
    bool cand = (double)x >= thr;
    unsigned long long k = key_of<T>(x);
    gt[i] = cand && k > kstar ? 1 : 0;
    eq[i] = cand && k == kstar ? 1 : 0;
}

__global__ void k_sel_final(int64_t moff, const int64_t *gt, const int64_t *eq,
                            const int64_t *eqrank, int64_t need, int64_t *flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < moff) flag[i] = gt[i] || (eq[i] && eqrank[i] < need) ? 1 : 0;
}

template <typename T>
static int64_t filter_T(grass_ctx_t ctx, grass_sparsifier_t S, const T *heat, double thr,
                        int64_t cap, int64_t *accepted) {
    const int64_t moff = S->m_off;
    if (moff == 0) return 0;
    int64_t *flag = ctx->scr<int64_t>(SCR_FILTER, moff + 1);
    int64_t *pos = ctx->scr<int64_t>(SCR_FILTER2, moff + 1);
    int64_t g = cdiv(moff, kBlock);
    launch(ctx, k_thr_flag<T>, g, kBlock, 0, moff, heat, thr, flag);
    int64_t count = 0;
    scan_i64(ctx, flag, pos, moff, &count);
    if (cap > 0 && count > cap) {
        // radix select of the cap-th largest key among the candidates
        unsigned int *hist = (unsigned int *)ctx->scr<char>(SCR_TMP2, 256 * sizeof(unsigned int));
        const int bits = (int)sizeof(T) * 8;
        unsigned long long prefix = 0, mask = 0;
        int64_t need = cap;
        unsigned int hh[256];
        int64_t hgrid = std::min<int64_t>(kRedBlocks, g);
        for (int shift = bits - 8; shift >= 0; shift -= 8) {
            memset_d(ctx, hist, 0, 256 * sizeof(unsigned int));
            launch(ctx, k_radix_hist<T>, hgrid, kBlock, 0, moff, heat, thr, prefix, mask, shift,
                   hist);
            d2h(ctx, hh, hist, sizeof(hh));
            int b = 255;
            for (; b >= 0; --b) {
                if ((int64_t)hh[b] >= need) break;
                need -= hh[b];
            }
            if (b < 0) fail(GRASS_ERR_CUDA, "radix select lost its candidates");
            prefix |= (unsigned long long)b << shift;
            mask |= 0xFFULL << shift;
        }
        int64_t *gt = ctx->scr<int64_t>(SCR_TMP0, moff + 1);
        int64_t *eq = ctx->scr<int64_t>(SCR_TMP1, moff + 1);
        int64_t *eqr = ctx->scr<int64_t>(SCR_TMP3, moff + 1);
        launch(ctx, k_sel_flags<T>, g, kBlock, 0, moff, heat, thr, prefix, gt, eq);
        scan_i64(ctx, eq, eqr, moff, nullptr);
        launch(ctx, k_sel_final, g, kBlock, 0, moff, (const int64_t *)gt, (const int64_t *)eq,
               (const int64_t *)eqr, need, flag);
        scan_i64(ctx, flag, pos, moff, &count);
    }
    launch(ctx, k_scatter_ids, g, kBlock, 0, moff, (const int64_t *)flag, (const int64_t *)pos,
           (const int32_t *)S->off_eid.p, accepted);
    return count;
}

int64_t filter_heat(grass_ctx_t ctx, grass_sparsifier_t S, const void *heat, grass_prec prec,
                    double thr, int64_t cap, int64_t *accepted) {
    if (prec == GRASS_FP64) return filter_T<double>(ctx, S, (const double *)heat, thr, cap, accepted);
    return filter_T<float>(ctx, S, (const float *)heat, thr, cap, accepted);
}

// ---------------------------------------------------------------- similarity check (Sec. IV-D step 6)
// The greedy pass over the selected edges in priority order (heat
// descending, id ascending) that keeps an edge unless an endpoint already
// carries a kept edge is a greedy matching under a strict total order.  It
// equals the result of rounds that keep, at once, every remaining edge that
// has the highest priority at both of its endpoints among the remaining
// edges there, then drop the remaining edges that touch a kept one: the
// highest-priority remaining edge is always kept, so the rounds end, and no
// round keeps an edge that the sequential pass would reject.  Per vertex the
// highest priority is an atomicMax on the heat's bit pattern (non-negative
// floats order like their bits) followed by an atomicMin on the id among
// edges of that heat; the result does not depend on timing.

enum : uint8_t { SIM_ALIVE = 0, SIM_KEPT = 1, SIM_DROPPED = 2 };

// candidates: off-S positions i with heat[i] >= thr (flag from k_thr_flag)
__global__ void k_sim_init(int64_t moff, const int64_t *flag, const int32_t *ou, const int32_t *ov,
                           uint8_t *state, unsigned long long *vbest, int32_t *vid, uint8_t *vmatched) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= moff) return;
    state[i] = flag[i] ? SIM_ALIVE : SIM_DROPPED;
    if (!flag[i]) return;
    const int32_t u = ou[i], v = ov[i];
    vbest[u] = 0ULL;
    vbest[v] = 0ULL;
    vid[u] = 0x7FFFFFFF;
    vid[v] = 0x7FFFFFFF;
    vmatched[u] = 0;
    vmatched[v] = 0;
}

template <typename T>
__global__ void k_sim_max(int64_t moff, const uint8_t *state, const T *heat, const int32_t *ou,
                          const int32_t *ov, unsigned long long *vbest) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= moff || state[i] != SIM_ALIVE) return;
    const unsigned long long k = key_of<T>(heat[i]);
    atomicMax(vbest + ou[i], k);
    atomicMax(vbest + ov[i], k);
}

template <typename T>
__global__ void k_sim_min(int64_t moff, const uint8_t *state, const T *heat, const int32_t *ou,
                          const int32_t *ov, const int32_t *oe, const unsigned long long *vbest,
                          int32_t *vid) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= moff || state[i] != SIM_ALIVE) return;
    const unsigned long long k = key_of<T>(heat[i]);
    if (vbest[ou[i]] == k) atomicMin(vid + ou[i], oe[i]);
    if (vbest[ov[i]] == k) atomicMin(vid + ov[i], oe[i]);
}

__global__ void k_sim_keep(int64_t moff, uint8_t *state, const int32_t *ou, const int32_t *ov,
                           const int32_t *oe, const int32_t *vid, uint8_t *vmatched) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= moff || state[i] != SIM_ALIVE) return;
    if (vid[ou[i]] == oe[i] && vid[ov[i]] == oe[i]) {
        state[i] = SIM_KEPT;
        vmatched[ou[i]] = 1;
        vmatched[ov[i]] = 1;
    }
}

// drop the remaining edges at a kept edge's endpoint, reset the per-vertex
// best for the next round and count the edges still remaining
__global__ void k_sim_prune(int64_t moff, uint8_t *state, const int32_t *ou, const int32_t *ov,
                            const uint8_t *vmatched, unsigned long long *vbest, int32_t *vid,
                            unsigned long long *alive) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool a = false;
    if (i < moff && state[i] == SIM_ALIVE) {
        const int32_t u = ou[i], v = ov[i];
        if (vmatched[u] || vmatched[v]) state[i] = SIM_DROPPED;
        else a = true;
        vbest[u] = 0ULL;
        vbest[v] = 0ULL;
        vid[u] = 0x7FFFFFFF;
        vid[v] = 0x7FFFFFFF;
    }
    const unsigned int cnt = __popc(__ballot_sync(0xffffffffu, a));
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(alive, (unsigned long long)cnt);
}

// heat of the kept edges, -1 (below any threshold) for the others
template <typename T>
__global__ void k_sim_heat(int64_t moff, const uint8_t *state, const T *heat, T *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < moff) out[i] = state[i] == SIM_KEPT ? heat[i] : (T)-1;
}

template <typename T>
static int64_t similar_T(grass_ctx_t ctx, grass_sparsifier_t S, const T *heat, double thr,
                         int64_t cap, int64_t *accepted) {
    const int64_t moff = S->m_off, n = S->tree->g.n;
    if (moff == 0) return 0;
    const int64_t g = cdiv(moff, kBlock);
    int64_t *flag = ctx->scr<int64_t>(SCR_FILTER, moff + 1);
    uint8_t *state = ctx->scr<uint8_t>(SCR_SIM_C, moff + 1);
    // per vertex: best key, best id, matched flag; one round's live count
    char *vb = ctx->scr<char>(SCR_SIM_V, (size_t)n * (8 + 4 + 1) + 64);
    unsigned long long *vbest = reinterpret_cast<unsigned long long *>(vb);
    int32_t *vid = reinterpret_cast<int32_t *>(vb + (size_t)n * 8);
    uint8_t *vmatched = reinterpret_cast<uint8_t *>(vb + (size_t)n * 12);
    unsigned long long *alive = reinterpret_cast<unsigned long long *>(ctx->scal.p + DS_MAX + 10);
    const int32_t *ou = S->off_u.p, *ov = S->off_v.p, *oe = S->off_eid.p;
    launch(ctx, k_thr_flag<T>, g, kBlock, 0, moff, heat, thr, flag);
    launch(ctx, k_sim_init, g, kBlock, 0, moff, (const int64_t *)flag, ou, ov, state, vbest, vid,
           vmatched);
    for (int64_t round = 0;; ++round) {
        if (round > moff) fail(GRASS_ERR_CUDA, "similarity check did not finish");
        launch(ctx, k_sim_max<T>, g, kBlock, 0, moff, (const uint8_t *)state, heat, ou, ov, vbest);
        launch(ctx, k_sim_min<T>, g, kBlock, 0, moff, (const uint8_t *)state, heat, ou, ov, oe,
               (const unsigned long long *)vbest, vid);
        launch(ctx, k_sim_keep, g, kBlock, 0, moff, state, ou, ov, oe, (const int32_t *)vid,
               vmatched);
        memset_d(ctx, alive, 0, sizeof(unsigned long long));
        launch(ctx, k_sim_prune, g, kBlock, 0, moff, state, ou, ov, (const uint8_t *)vmatched,
               vbest, vid, alive);
        unsigned long long left = 0;
        d2h(ctx, &left, alive, sizeof(left));
        if (left == 0) break;
    }
    T *kept_heat = reinterpret_cast<T *>(ctx->scr<char>(SCR_SIM_E, (size_t)(moff + 1) * sizeof(T)));
    launch(ctx, k_sim_heat<T>, g, kBlock, 0, moff, (const uint8_t *)state, heat, kept_heat);
    return filter_T<T>(ctx, S, kept_heat, thr, cap, accepted);
}

int64_t filter_similar(grass_ctx_t ctx, grass_sparsifier_t S, const void *heat, grass_prec prec,
                       double thr, int64_t cap, int64_t *accepted) {
    if (prec == GRASS_FP64) return similar_T<double>(ctx, S, (const double *)heat, thr, cap, accepted);
    return similar_T<float>(ctx, S, (const float *)heat, thr, cap, accepted);
}

}  // namespace grass
