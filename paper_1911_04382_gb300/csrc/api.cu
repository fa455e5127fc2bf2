// api.cu -- the extern "C" entry points declared in include/grass.h:
// argument checks, orchestration of the kernels of the other files, the
// power iteration (Sec. III-F), the lambda estimates (Sec. IV-C) and the
// densification loop (Sec. IV-D).
#include <chrono>
#include <cmath>
#include <new>

#include "common.cuh"

using namespace grass;

#define API_BEGIN(ctx)                                                   \
    grass_ctx_t api_ctx_ = (ctx);                                        \
    try {                                                                \
        if (api_ctx_) GCK(cudaSetDevice(api_ctx_->device));
#define API_END                                                          \
    }                                                                    \
    catch (const grass::Error &e) {                                      \
        if (api_ctx_) api_ctx_->err = e.msg;                             \
        return e.st;                                                     \
    }                                                                    \
    catch (const std::bad_alloc &) {                                     \
        if (api_ctx_) api_ctx_->err = "host allocation failed";          \
        return GRASS_ERR_OOM;                                            \
    }                                                                    \
    catch (...) {                                                        \
        if (api_ctx_) api_ctx_->err = "unexpected internal error";       \
        return GRASS_ERR_CUDA;                                           \
    }                                                                    \
    return GRASS_OK;

namespace grass {

// ---------------------------------------------------------------- helpers
// (shared with the batch entry points of batch.cu)

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t esize(grass_prec p) { return p == GRASS_FP64 ? 8 : 4; }

void need(bool ok, const char *msg) {
    if (!ok) fail(GRASS_ERR_INVALID, msg);
}

void need_prec(grass_prec p) { need(p == GRASS_FP64 || p == GRASS_FP32, "prec must be GRASS_FP64 or GRASS_FP32"); }

unsigned long long *maxslot(grass_ctx_t ctx, int k) {
    return (unsigned long long *)(ctx->scal.p + DS_MAX) + k;
}

double bits_to_double(unsigned long long b) {
    double d;
    std::memcpy(&d, &b, sizeof(d));
    return d;
}

// A bounded device wait that ran out leaves flags[3] set: report it and
// clear it for the next call.
void clear_timeout(grass_ctx_t ctx) { memset_d(ctx, ctx->flags.p + 3, 0, sizeof(int)); }

void check_timeout(grass_ctx_t ctx) {
    int f = 0;
    d2h(ctx, &f, ctx->flags.p + 3, sizeof(int));
    if (f) {
        clear_timeout(ctx);
        ctx->sync();
        fail(GRASS_ERR_TIMEOUT, "a bounded device-side wait expired (grid barrier)");
    }
}

void ensure_sdd(grass_ctx_t ctx, grass_tree_t T) {
    if (!T->has_sdd) {
        tree_factor(ctx, T, true, T->sdd);
        T->has_sdd = true;
    }
}

// Sec. III-F, Eq. (formula_pwr_iter): t steps H <- L_S^{-1} L_G H.  H holds
// the unscaled last iterate on return; *scale_slot the max-abs bits that
// give its pending power-of-two factor.  Returns inner CG iterations.
// stop_when_capped ends the steps after the first inner solve that reached
// inner_maxit (the DS_CAPPED counter, zeroed by the caller).
static int64_t power_steps_until(grass_ctx_t ctx, grass_sparsifier_t S, const double *h0, int r,
                                 int t, grass_prec prec, double inner_tol, int inner_maxit,
                                 void *H, void *Y, int *scale_slot, bool stop_when_capped) {
    const GraphData &g = S->tree->g;
    const int64_t n = g.n;
    convert_block(ctx, prec, n * r, h0, H);
    const void *w = prec == GRASS_FP64 ? (const void *)g.adj_w64.p : (const void *)g.adj_w32.p;
    int prev = -1, cur = 0;
    int64_t inner = 0;
    for (int s = 0; s < t; ++s) {
        lap_mm(ctx, r, prec, n, 2 * g.m, g.adj_ptr.p, g.adj_col.p, w, nullptr, H, Y,
               prev >= 0 ? maxslot(ctx, prev) : nullptr, GRASS_KF_SPMM_G, &g.heavy);
        memset_d(ctx, maxslot(ctx, cur), 0, sizeof(unsigned long long));
        inner += s_solve(ctx, S, false, r, prec, Y, H, inner_tol, inner_maxit, maxslot(ctx, cur));
        prev = cur;
        cur ^= 1;
        if (stop_when_capped && !S->is_tree && s + 1 < t) {
            // the caller's counter of solves that reached inner_maxit
            double capped = 0.0;
            d2h(ctx, &capped, ctx->scal.p + DS_RED + DS_CAPPED, sizeof(double));
            if (capped > 0.0) break;
        }
    }
    *scale_slot = prev;
    return inner;
}

int64_t power_steps(grass_ctx_t ctx, grass_sparsifier_t S, const double *h0, int r, int t,
                    grass_prec prec, double inner_tol, int inner_maxit, void *H, void *Y,
                    int *scale_slot) {
    return power_steps_until(ctx, S, h0, r, t, prec, inner_tol, inner_maxit, H, Y, scale_slot,
                             false);
}

struct EmbedOut {
    double heat_max;
    int64_t inner;
};

EmbedOut embed_impl(grass_ctx_t ctx, grass_sparsifier_t S, const double *h0, int r, int t,
                    grass_prec prec, double inner_tol, int inner_maxit, void *H_out, void *heat) {
    const int64_t n = S->tree->g.n;
    void *H = ctx->scr<char>(SCR_H, n * r * esize(prec));
    void *Y = ctx->scr<char>(SCR_Y, n * r * esize(prec));
    int slot = 0;
    EmbedOut o{0.0, 0};
    o.inner = power_steps(ctx, S, h0, r, t, prec, inner_tol, inner_maxit, H, Y, &slot);
    unsigned long long *hm = maxslot(ctx, 2);
    heat_offs(ctx, r, prec, S, H, maxslot(ctx, slot), heat, hm);
    if (H_out) {
        copy_d(ctx, H_out, H, n * r * esize(prec));
        apply_pow2(ctx, prec, n * r, H_out, maxslot(ctx, slot));
    }
    unsigned long long b = 0;
    d2h(ctx, &b, hm, sizeof(b));
    o.heat_max = bits_to_double(b);
    return o;
}

// Sec. IV-C-1: iters generalized power steps, then v^T L_G v / v^T L_S v.
// stop_when_capped: end the steps after the first inner solve that reached
// inner_maxit; the quotient is then taken on that step's vector.
double lambda_max_impl(grass_ctx_t ctx, grass_sparsifier_t S, const double *v0, int iters,
                       grass_prec prec, double inner_tol, int inner_maxit, int64_t *inner,
                       bool stop_when_capped) {
    const int64_t n = S->tree->g.n;
    void *v = ctx->scr<char>(SCR_LMAX_V, n * esize(prec));
    void *y = ctx->scr<char>(SCR_LMAX_Y, n * esize(prec));
    int slot = -1;
    if (iters > 0) {
        *inner += power_steps_until(ctx, S, v0, 1, iters, prec, inner_tol, inner_maxit, v, y,
                                    &slot, stop_when_capped);
        apply_pow2(ctx, prec, n, v, maxslot(ctx, slot));
    } else {
        convert_block(ctx, prec, n, v0, v);
    }
    double *q = ctx->scal.p + DS_RED + 16;
    quad_forms(ctx, prec, S, v, q);
    double qq[2];
    d2h(ctx, qq, q, sizeof(qq));
    check_timeout(ctx);   // a solve that gave up leaves garbage: report that first
    if (!(qq[1] > 0.0)) fail(GRASS_ERR_INVALID, "v^T L_S v is not positive (v0 constant?)");
    return qq[0] / qq[1];
}

double theta_sigma(double sigma2, double lmin, double lmax, int t) {
    // Eq. (formula_heatratio_final)
    return std::pow(sigma2 * lmin / lmax, 2 * t + 1);
}

grass_sparsifier_t new_sparsifier(grass_ctx_t ctx, grass_tree_t T) {
    auto *S = new grass_sparsifier_s();
    S->ctx = ctx;
    S->tree = T;
    try {
        S->in_s.alloc(T->g.m);
        copy_d(ctx, S->in_s.p, T->in_tree.p, T->g.m);
        sparsifier_rebuild(ctx, S);
    } catch (...) {
        delete S;
        throw;
    }
    return S;
}

__global__ void k_mark_roots(int64_t nroots, const int32_t *roots, uint8_t *isroot) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nroots) isroot[roots[q]] = 1;
}

// ---------------------------------------------------------------- a caller's tree

__global__ void k_user_mark(int64_t cnt, const int64_t *eids, int64_t m, uint8_t *in_tree,
                            int *bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int64_t e = eids[i];
    if (e < 0 || e >= m) {
        atomicOr(bad, 1);
        return;
    }
    in_tree[e] = 1;
}

// w[e] = 2 for the caller's edges, 1 for the others: the maximum spanning
// tree under these weights contains every caller edge unless they close a
// cycle
__global__ void k_indicator_w(int64_t m, const uint8_t *mark, double *w) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) w[e] = mark[e] ? 2.0 : 1.0;
}

// counts[0] += #{e : a[e] != 0}, counts[1] += #{e : a[e] != b[e]}
__global__ void k_mask_counts(int64_t m, const uint8_t *a, const uint8_t *b,
                              unsigned long long *counts) {
    unsigned long long ones = 0, diff = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        ones += a[e] != 0;
        diff += (a[e] != 0) != (b[e] != 0);
    }
    for (int d = 16; d > 0; d >>= 1) {
        ones += __shfl_xor_sync(0xffffffffu, ones, d);
        diff += __shfl_xor_sync(0xffffffffu, diff, d);
    }
    if ((threadIdx.x & 31) == 0) {
        if (ones) atomicAdd(counts, ones);
        if (diff) atomicAdd(counts + 1, diff);
    }
}

// in_tree = the caller's n-1 edge ids, after checking that they are a
// spanning tree of the graph: ids in range and distinct, and equal to the
// maximum spanning tree under weights that prefer them (which holds iff
// they contain no cycle; n-1 acyclic edges of a connected graph span it).
void user_tree(grass_ctx_t ctx, const GraphData &g, const int64_t *eids, uint8_t *in_tree) {
    const int64_t n = g.n, m = g.m;
    memset_d(ctx, in_tree, 0, (size_t)m);
    memset_d(ctx, ctx->flags.p, 0, sizeof(int));
    launch(ctx, k_user_mark, cdiv(n - 1, kBlock), kBlock, 0, n - 1, eids, m, in_tree,
           ctx->flags.p);
    int bad = 0;
    d2h(ctx, &bad, ctx->flags.p, sizeof(int));
    if (bad) fail(GRASS_ERR_INVALID, "tree edge id out of range");
    DBuf<double> w;
    w.alloc(m);
    DBuf<uint8_t> chk;
    chk.alloc(m);
    DBuf<unsigned long long> cnt;
    cnt.alloc(2);
    launch(ctx, k_indicator_w, cdiv(m, kBlock), kBlock, 0, m, (const uint8_t *)in_tree, w.p);
    mst_boruvka_w(ctx, g, w.p, chk.p);
    memset_d(ctx, cnt.p, 0, 2 * sizeof(unsigned long long));
    launch(ctx, k_mask_counts, std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, cdiv(m, kBlock))),
           kBlock, 0, m, (const uint8_t *)in_tree, (const uint8_t *)chk.p, cnt.p);
    unsigned long long c[2] = {0, 0};
    d2h(ctx, c, cnt.p, sizeof(c));
    if ((int64_t)c[0] != n - 1)
        fail(GRASS_ERR_INVALID, "tree edge ids are not distinct (" + std::to_string(c[0]) +
                                    " distinct edges for n - 1 = " + std::to_string(n - 1) + ")");
    if (c[1] != 0) fail(GRASS_ERR_INVALID, "the tree edges contain a cycle (they do not span the graph)");
}

// Spanning tree (one root) or spanning forest of a batch (one root per graph,
// the graph's first vertex), its elimination schedule and the L_T factor.
// user_eids (device, n-1 edge ids) replaces the maximum spanning tree by the
// caller's tree, lsst_seed by the low-stretch tree of that seed (single graph
// only).
grass_tree_t build_tree_impl(grass_ctx_t ctx, const grass_csr_t *A,
                             const std::vector<int64_t> &voff, const std::vector<int32_t> &roots,
                             const int64_t *user_eids = nullptr, const uint64_t *lsst_seed = nullptr,
                             LsstStats *lsst_stats = nullptr) {
    auto *T = new grass_tree_s();
    T->ctx = ctx;
    T->nroots = (int64_t)roots.size();
    T->roots_h = roots;
    T->ground = roots[0];
    T->g.nseg = (int64_t)roots.size();
    if (T->g.nseg > 1) T->g.seg_voff = voff;
    try {
        graph_extract(ctx, A, T->g);
        const int64_t n = T->g.n;
        T->roots.alloc(T->nroots);
        h2d(ctx, T->roots.p, roots.data(), roots.size() * sizeof(int32_t));
        T->isroot.alloc(n);
        memset_d(ctx, T->isroot.p, 0, n);
        launch(ctx, k_mark_roots, cdiv(T->nroots, kBlock), kBlock, 0, T->nroots,
               (const int32_t *)T->roots.p, T->isroot.p);
        T->in_tree.alloc(T->g.m);
        if (user_eids) user_tree(ctx, T->g, user_eids, T->in_tree.p);
        else if (lsst_seed) lsst_build(ctx, T->g, *lsst_seed, T->in_tree.p, lsst_stats);
        else mst_boruvka(ctx, T->g, T->in_tree.p);
        tree_schedule(ctx, T);
        tree_factor(ctx, T, false, T->lap);
        ctx->sync();
    } catch (...) {
        delete T;
        throw;
    }
    return T;
}

}  // namespace grass

extern "C" {

// ---------------------------------------------------------------- context

grass_status grass_ctx_create(grass_ctx_t *out, void *stream) {
    if (!out) return GRASS_ERR_INVALID;
    *out = nullptr;
    grass_ctx_t ctx = nullptr;
    try {
        int dev = 0;
        int count = 0;
        GCK(cudaGetDeviceCount(&count));
        if (count <= 0) fail(GRASS_ERR_CUDA, "no CUDA device");
        GCK(cudaGetDevice(&dev));
        ctx = new grass_ctx_s();
        ctx->device = dev;
        ctx->stream = (cudaStream_t)stream;
        ctx->flags.alloc(8);
        ctx->scal.alloc(DS_TOTAL);
        ctx->partials.alloc((size_t)kRedBlocks * 32 * 2);
        ctx->counters.alloc(16);
        GCK(cudaMemset(ctx->counters.p, 0, 16 * sizeof(unsigned int)));
        GCK(cudaMemset(ctx->flags.p, 0, 8 * sizeof(int)));
        GCK(cudaMemset(ctx->scal.p, 0, DS_TOTAL * sizeof(double)));
        GCK(cudaMallocHost((void **)&ctx->hpin, 4096 * sizeof(double)));
        ctx->gbar.alloc(4);
        GCK(cudaMemset(ctx->gbar.p, 0, 4 * sizeof(unsigned int)));
        int coop = 0, sms = 0;
        GCK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        GCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        ctx->num_sms = coop ? sms : 0;   // 0: per-round launches instead of one cooperative kernel
        GCK(cudaDeviceSynchronize());
    } catch (const grass::Error &e) {
        delete ctx;
        return e.st;
    } catch (...) {
        delete ctx;
        return GRASS_ERR_CUDA;
    }
    *out = ctx;
    return GRASS_OK;
}

void grass_ctx_destroy(grass_ctx_t ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->hpin) cudaFreeHost(ctx->hpin);
    delete ctx;
}

grass_status grass_ctx_set_stream(grass_ctx_t ctx, void *stream) {
    if (!ctx) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    ctx->sync();
    ctx->stream = (cudaStream_t)stream;
    API_END
}

const char *grass_last_error(grass_ctx_t ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t grass_launch_count(grass_ctx_t ctx) { return ctx ? ctx->launches : 0; }

grass_status grass_ctx_set_wait_limit(grass_ctx_t ctx, int64_t polls, int hold_barriers) {
    if (!ctx) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(polls >= 0, "polls must be >= 0");
    ctx->wait_budget = polls > 0 ? (long long)polls : (1LL << 23);
    unsigned int h = hold_barriers ? 1u : 0u;
    GCK(cudaMemcpyAsync(ctx->gbar.p + 2, &h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
    ctx->sync();
    API_END
}

grass_status grass_ctx_set_param(grass_ctx_t ctx, const char *name, int64_t value) {
    if (!ctx || !name) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    std::string k(name);
    if (k == "tree_blocks_per_sm") {
        need(value >= 1 && value <= 8, "tree_blocks_per_sm must be in [1, 8]");
        ctx->tree_bpsm = (int)value;
    } else if (k == "tree_threads") {
        need(value >= 128 && value <= kPersistMaxThreads && value % 32 == 0,
             "tree_threads must be a multiple of 32 in [128, 1024]");
        ctx->tree_threads = (int)value;
    } else if (k == "tree_tail_items") {
        need(value >= 0, "tree_tail_items must be >= 0");
        ctx->tree_tail_items = value;
    } else if (k == "euler_solve") {
        need(value == 0 || value == 1, "euler_solve must be 0 or 1");
        ctx->euler_solve = (int)value;
    } else if (k == "similarity_check") {
        need(value == 0 || value == 1, "similarity_check must be 0 or 1");
        ctx->similarity_check = (int)value;
    } else if (k == "pcg_precond") {
        need(value == 0 || value == 1, "pcg_precond must be 0 or 1");
        ctx->pcg_precond = (int)value;
    } else if (k == "amg_sweeps") {
        need(value >= 1 && value <= 8, "amg_sweeps must be in [1, 8]");
        ctx->amg_sweeps = (int)value;
    } else if (k == "amg_fused") {
        need(value == 0 || value == 1, "amg_fused must be 0 or 1");
        ctx->amg_fused = (int)value;
    } else if (k == "amg_warp_n") {
        need(value >= 0, "amg_warp_n must be >= 0");
        ctx->amg_warp_n = value;
    } else if (k == "amg_warp_setup_n") {
        need(value >= 0, "amg_warp_setup_n must be >= 0");
        ctx->amg_warp_setup_n = value;
    } else if (k == "amg_tail_n") {
        need(value >= 0, "amg_tail_n must be >= 0");
        ctx->amg_tail_n = value;
    } else if (k == "lmax_amg") {
        need(value == 0 || value == 1, "lmax_amg must be 0 or 1");
        ctx->lmax_amg = (int)value;
    } else if (k == "spmm_variant") {
        need(value >= -1 && value <= 7, "spmm_variant must be in [-1, 7]");
        ctx->spmm_variant = (int)value;
    } else if (k == "spmm_chunk") {
        need(value == -1 || value == 0 || value == 16, "spmm_chunk must be -1, 0 or 16");
        ctx->spmm_chunk = (int)value;
    } else if (k == "lsst_small_level") {
        need(value >= 0, "lsst_small_level must be >= 0");
        ctx->lsst_small_level = value;
    } else if (k == "heat_lanes") {
        need(value >= 0 && value <= 3, "heat_lanes must be in [0, 3]");
        ctx->heat_lanes = (int)value;
    } else if (k == "grid_sms") {
        need(value >= 0, "grid_sms must be >= 0");
        ctx->grid_sms = (int)value;
    } else if (k == "euler_max_n") {
        need(value >= 0, "euler_max_n must be >= 0");
        ctx->euler_max_n = value;
    } else {
        fail(GRASS_ERR_INVALID, "unknown parameter " + k);
    }
    API_END
}

grass_status grass_tree_schedule_info(grass_tree_t T, int64_t *eliminated, int64_t *receivers,
                                      int64_t *contributions, int64_t cap) {
    if (!T || cap < 0) return GRASS_ERR_INVALID;
    const TreeSchedule &S = T->sched;
    for (int k = 0; k < S.rounds && k < cap; ++k) {
        if (eliminated) eliminated[k] = S.elim_off[k + 1] - S.elim_off[k];
        if (receivers) receivers[k] = S.rcv_off[k + 1] - S.rcv_off[k];
        if (contributions) {
            contributions[k] = 0;   // filled below from the host offsets
        }
    }
    if (contributions) {
        // contributions of round k = rcv_beg[rcv_off[k+1]] - rcv_beg[rcv_off[k]]
        std::vector<int32_t> beg(S.n_rcv + 1);
        if (cudaMemcpy(beg.data(), S.rcv_beg.p, beg.size() * sizeof(int32_t),
                       cudaMemcpyDeviceToHost) != cudaSuccess)
            return GRASS_ERR_CUDA;
        for (int k = 0; k < S.rounds && k < cap; ++k)
            contributions[k] = beg[S.rcv_off[k + 1]] - beg[S.rcv_off[k]];
    }
    return GRASS_OK;
}

grass_status grass_kernel_timing_enable(grass_ctx_t ctx, int family) {
    if (!ctx) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(family >= GRASS_KF_NONE && family <= GRASS_KF_SPMM_BLK, "unknown kernel family");
    ctx->sync();
    ctx->tfam = family;
    ctx->ev_used = 0;
    ctx->t_launches = 0;
    ctx->t_bytes = 0.0;
    ctx->iter_launches.clear();
    API_END
}

grass_status grass_kernel_timing_read(grass_ctx_t ctx, double *ms, int64_t *launches,
                                      double *bytes) {
    if (!ctx) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    ctx->sync();
    double tot = 0.0;
    for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
        float e = 0.f;
        GCK(cudaEventElapsedTime(&e, ctx->events[i], ctx->events[i + 1]));
        tot += e;
    }
    double by = ctx->t_bytes;
    if (!ctx->iter_launches.empty()) {
        std::vector<double> snap(2 * ctx->iter_launches.size());
        d2h(ctx, snap.data(), ctx->iter_snap.p, snap.size() * sizeof(double));
        for (const auto &l : ctx->iter_launches)
            by += l.fixed + l.per_iter * (snap[2 * l.slot + 1] - snap[2 * l.slot]);
    }
    if (ms) *ms = tot;
    if (launches) *launches = ctx->t_launches;
    if (bytes) *bytes = by;
    API_END
}

// ---------------------------------------------------------------- tree

grass_status grass_build_tree(grass_ctx_t ctx, const grass_csr_t *A, int32_t ground,
                              grass_tree_t *out) {
    if (!ctx) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(A && out, "null argument");
    *out = nullptr;
    need(ground >= 0 && ground < A->n, "ground must be in [0, n)");
    *out = build_tree_impl(ctx, A, {0, A->n}, {ground});
    API_END
}

grass_status grass_tree_from_edges(grass_ctx_t ctx, const grass_csr_t *A, const int64_t *tree_eids,
                                   int32_t ground, grass_tree_t *out) {
    if (!ctx) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(A && out && tree_eids, "null argument");
    *out = nullptr;
    need(ground >= 0 && ground < A->n, "ground must be in [0, n)");
    *out = build_tree_impl(ctx, A, {0, A->n}, {ground}, tree_eids);
    API_END
}

grass_status grass_build_lsst(grass_ctx_t ctx, const grass_csr_t *A, uint64_t seed, int32_t ground,
                              grass_tree_t *out, grass_lsst_stats_t *stats) {
    if (!ctx) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(A && out, "null argument");
    *out = nullptr;
    need(ground >= 0 && ground < A->n, "ground must be in [0, n)");
    LsstStats ls;
    cudaEvent_t ev[2];
    GCK(cudaEventCreate(&ev[0]));
    GCK(cudaEventCreate(&ev[1]));
    GCK(cudaEventRecord(ev[0], ctx->stream));
    try {
        *out = build_tree_impl(ctx, A, {0, A->n}, {ground}, nullptr, &seed, &ls);
    } catch (...) {
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        throw;
    }
    GCK(cudaEventRecord(ev[1], ctx->stream));
    GCK(cudaEventSynchronize(ev[1]));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (stats) {
        stats->classes = ls.classes;
        stats->levels = ls.levels;
        stats->rounds = ls.rounds;
        stats->ms = ms;
    }
    API_END
}

grass_status grass_autotune_rows(grass_ctx_t ctx, grass_tree_t tree, int r, grass_prec prec,
                                 int32_t *best, double *best_ms) {
    if (!ctx || !tree) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(r_supported(r), "r must be 1, 2, 4, 8, 16, 24 or 32");
    need_prec(prec);
    autotune_rows(ctx, tree, r, prec, best, best_ms);
    API_END
}

grass_status grass_tree_stretch(grass_ctx_t ctx, grass_tree_t tree, double *stretch, double *total) {
    if (!ctx || !tree) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(tree->ctx == ctx, "tree belongs to another context");
    need(tree->nroots == 1, "stretch is defined here for a single spanning tree");
    tree_stretch(ctx, tree, stretch, total);
    API_END
}

grass_status grass_build_forest(grass_ctx_t ctx, const grass_csr_t *A, int64_t nseg,
                                const int64_t *seg_off, grass_tree_t *out) {
    if (!ctx) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(A && out && seg_off, "null argument");
    *out = nullptr;
    need(nseg >= 1 && nseg <= (1 << 20), "nseg must be in [1, 2^20]");
    need(seg_off[0] == 0 && seg_off[nseg] == A->n, "seg_off must start at 0 and end at n");
    std::vector<int64_t> voff(seg_off, seg_off + nseg + 1);
    std::vector<int32_t> roots(nseg);
    for (int64_t k = 0; k < nseg; ++k) {
        need(voff[k + 1] - voff[k] >= 2, "every graph of the batch needs at least 2 vertices");
        roots[k] = (int32_t)voff[k];
    }
    *out = build_tree_impl(ctx, A, voff, roots);
    API_END
}

grass_status grass_tree_segments(grass_tree_t T, int64_t *nseg, int64_t *vtx_off,
                                 int64_t *edge_off) {
    if (!T) return GRASS_ERR_INVALID;
    const GraphData &g = T->g;
    if (nseg) *nseg = g.nseg;
    if (vtx_off) std::copy(g.seg_voff.begin(), g.seg_voff.end(), vtx_off);
    if (edge_off) std::copy(g.seg_eoff.begin(), g.seg_eoff.end(), edge_off);
    return GRASS_OK;
}

void grass_tree_destroy(grass_tree_t T) {
    if (!T) return;
    cudaSetDevice(T->ctx->device);
    delete T;
}

grass_status grass_tree_info(grass_tree_t T, int64_t *n, int64_t *m, int64_t *rounds) {
    if (!T) return GRASS_ERR_INVALID;
    if (n) *n = T->g.n;
    if (m) *m = T->g.m;
    if (rounds) *rounds = T->sched.rounds;
    return GRASS_OK;
}

grass_status grass_tree_graph(grass_ctx_t ctx, grass_tree_t T, int32_t *eu, int32_t *ev,
                              double *ew, double *D) {
    if (!ctx || !T) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    const int64_t m = T->g.m, n = T->g.n;
    if (eu) copy_d(ctx, eu, T->g.eu.p, m * sizeof(int32_t));
    if (ev) copy_d(ctx, ev, T->g.ev.p, m * sizeof(int32_t));
    if (ew) copy_d(ctx, ew, T->g.ew64.p, m * sizeof(double));
    if (D) copy_d(ctx, D, T->g.D64.p, n * sizeof(double));
    ctx->sync();
    API_END
}

grass_status grass_tree_edges(grass_ctx_t ctx, grass_tree_t T, uint8_t *in_tree) {
    if (!ctx || !T) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(in_tree, "null output");
    copy_d(ctx, in_tree, T->in_tree.p, T->g.m);
    ctx->sync();
    API_END
}

grass_status grass_tree_solve(grass_ctx_t ctx, grass_tree_t T, int with_D, int r,
                              grass_prec prec, const void *B, void *X) {
    if (!ctx || !T) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(B && X, "null block");
    need_prec(prec);
    need(r_supported(r), "r must be 1, 2, 4, 8, 16, 24 or 32");
    if (with_D) ensure_sdd(ctx, T);
    if (X != B) copy_d(ctx, X, B, T->g.n * r * esize(prec));
    clear_timeout(ctx);
    tree_solve_inplace(ctx, T, with_D ? T->sdd : T->lap, r, prec, X, nullptr);
    check_timeout(ctx);
    API_END
}

grass_status grass_spmm(grass_ctx_t ctx, grass_tree_t T, int r, grass_prec prec, const void *X,
                        void *Y) {
    if (!ctx || !T) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(X && Y && X != Y, "X, Y must be non-null and distinct");
    need_prec(prec);
    need(r_supported(r), "r must be 1, 2, 4, 8, 16, 24 or 32");
    const GraphData &g = T->g;
    lap_mm(ctx, r, prec, g.n, 2 * g.m, g.adj_ptr.p, g.adj_col.p,
           prec == GRASS_FP64 ? (const void *)g.adj_w64.p : (const void *)g.adj_w32.p, nullptr, X,
           Y, nullptr, GRASS_KF_SPMM_G, &g.heavy);
    API_END
}

// ---------------------------------------------------------------- sparsifier

grass_status grass_sparsifier_create(grass_ctx_t ctx, grass_tree_t T, grass_sparsifier_t *out) {
    if (!ctx || !T || !out) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    *out = nullptr;
    *out = new_sparsifier(ctx, T);
    ctx->sync();
    API_END
}

void grass_sparsifier_destroy(grass_sparsifier_t S) {
    if (!S) return;
    cudaSetDevice(S->ctx->device);
    delete S;
}

grass_status grass_sparsifier_add(grass_ctx_t ctx, grass_sparsifier_t S, const int64_t *eids,
                                  int64_t count) {
    if (!ctx || !S) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(count == 0 || eids, "null ids");
    sparsifier_add(ctx, S, eids, count);
    ctx->sync();
    API_END
}

grass_status grass_sparsifier_info(grass_sparsifier_t S, int64_t *n_edges, int64_t *m_off) {
    if (!S) return GRASS_ERR_INVALID;
    if (n_edges) *n_edges = S->n_edges;
    if (m_off) *m_off = S->m_off;
    return GRASS_OK;
}

grass_status grass_sparsifier_mask(grass_ctx_t ctx, grass_sparsifier_t S, uint8_t *in_s) {
    if (!ctx || !S) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(in_s, "null output");
    copy_d(ctx, in_s, S->in_s.p, S->tree->g.m);
    ctx->sync();
    API_END
}

__global__ void k_i32_to_i64(int64_t n, const int32_t *a, int64_t *b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

__global__ void k_s_flag(int64_t m, const uint8_t *in_s, int64_t *flag) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) flag[e] = in_s[e] ? 1 : 0;
}

__global__ void k_s_ids(int64_t m, const uint8_t *in_s, const int64_t *pos, int64_t *ids) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m && in_s[e]) ids[pos[e]] = e;
}

grass_status grass_sparsifier_edges(grass_sparsifier_t S, int64_t *eids_host, int64_t cap,
                                    int64_t *count) {
    if (!S || !count || cap < 0 || (cap > 0 && !eids_host)) return GRASS_ERR_INVALID;
    grass_ctx_t ctx = S->ctx;
    API_BEGIN(ctx)
    const int64_t m = S->tree->g.m;
    int64_t *flag = ctx->scr<int64_t>(SCR_TMP0, m + 1);
    int64_t *pos = ctx->scr<int64_t>(SCR_TMP1, m + 1);
    int64_t *ids = ctx->scr<int64_t>(SCR_TMP2, m + 1);
    launch(ctx, k_s_flag, cdiv(m, kBlock), kBlock, 0, m, (const uint8_t *)S->in_s.p, flag);
    int64_t ns = 0;
    scan_i64(ctx, flag, pos, m, &ns);
    launch(ctx, k_s_ids, cdiv(m, kBlock), kBlock, 0, m, (const uint8_t *)S->in_s.p,
           (const int64_t *)pos, ids);
    const int64_t k = std::min(cap, ns);
    if (k > 0) d2h(ctx, eids_host, ids, (size_t)k * sizeof(int64_t));
    ctx->sync();
    *count = ns;
    API_END
}

grass_status grass_sparsifier_offtree(grass_ctx_t ctx, grass_sparsifier_t S, int64_t *eids) {
    if (!ctx || !S) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(eids || S->m_off == 0, "null output");
    launch(ctx, k_i32_to_i64, cdiv(S->m_off, kBlock), kBlock, 0, S->m_off,
           (const int32_t *)S->off_eid.p, eids);
    ctx->sync();
    API_END
}

// ---------------------------------------------------------------- embed / filter

grass_status grass_embed(grass_ctx_t ctx, grass_sparsifier_t S, const double *h0, int r, int t,
                         grass_prec prec, double inner_tol, int inner_maxit, void *H_out,
                         void *heat, double *heat_max) {
    if (!ctx || !S) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(h0 != nullptr, "null h0");
    need_prec(prec);
    need(r_supported(r), "r must be 1, 2, 4, 8, 16, 24 or 32");
    need(t >= 1, "t must be >= 1");
    need(inner_maxit >= 0, "inner_maxit must be >= 0");
    void *hb = heat ? heat : (void *)ctx->scr<char>(SCR_HEAT, (S->m_off + 1) * esize(prec));
    clear_timeout(ctx);
    EmbedOut o = embed_impl(ctx, S, h0, r, t, prec, inner_tol, inner_maxit, H_out, hb);
    check_timeout(ctx);
    if (heat_max) *heat_max = o.heat_max;
    API_END
}

grass_status grass_lambda_min(grass_ctx_t ctx, grass_sparsifier_t S, double *lmin) {
    if (!ctx || !S || !lmin) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(S->tree->g.nseg == 1, "a batch of graphs: use grass_densify_batch");
    lambda_min(ctx, S, lmin);
    API_END
}

grass_status grass_lambda_max(grass_ctx_t ctx, grass_sparsifier_t S, const double *v0, int iters,
                              grass_prec prec, double inner_tol, int inner_maxit, double *lmax) {
    if (!ctx || !S || !lmax) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(S->tree->g.nseg == 1, "a batch of graphs: use grass_densify_batch");
    need(v0 != nullptr, "null v0");
    need_prec(prec);
    need(iters >= 0, "iters must be >= 0");
    int64_t inner = 0;
    clear_timeout(ctx);
    *lmax = lambda_max_impl(ctx, S, v0, iters, prec, inner_tol, inner_maxit, &inner, false);
    check_timeout(ctx);
    API_END
}

grass_status grass_filter(grass_ctx_t ctx, grass_sparsifier_t S, const void *heat, grass_prec prec,
                          double sigma2, double lmin, double lmax, int t, int64_t cap,
                          int64_t *accepted, int64_t *n_accepted, double *theta) {
    if (!ctx || !S || !n_accepted) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(S->tree->g.nseg == 1, "a batch of graphs: use grass_densify_batch");
    need(heat || S->m_off == 0, "null heat");
    need(accepted || S->m_off == 0, "null output");
    need_prec(prec);
    need(sigma2 > 0 && lmin > 0 && lmax > 0 && t >= 1, "sigma2, lmin, lmax must be > 0, t >= 1");
    double th = theta_sigma(sigma2, lmin, lmax, t);
    if (theta) *theta = th;
    *n_accepted = 0;
    if (S->m_off > 0) {
        unsigned long long *hm = maxslot(ctx, 3);
        memset_d(ctx, hm, 0, sizeof(unsigned long long));
        max_abs_bits(ctx, prec, S->m_off, heat, hm);
        unsigned long long b = 0;
        d2h(ctx, &b, hm, sizeof(b));
        double thr = th * bits_to_double(b);
        *n_accepted = filter_heat(ctx, S, heat, prec, thr, cap, accepted);
        ctx->sync();
    }
    API_END
}

grass_status grass_filter_similar(grass_ctx_t ctx, grass_sparsifier_t S, const void *heat,
                                  grass_prec prec, double sigma2, double lmin, double lmax, int t,
                                  int64_t cap, int64_t *accepted, int64_t *n_accepted,
                                  double *theta) {
    if (!ctx || !S || !n_accepted) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(S->tree->g.nseg == 1, "a batch of graphs: use grass_densify_batch");
    need(heat || S->m_off == 0, "null heat");
    need(accepted || S->m_off == 0, "null output");
    need_prec(prec);
    need(sigma2 > 0 && lmin > 0 && lmax > 0 && t >= 1, "sigma2, lmin, lmax must be > 0, t >= 1");
    double th = theta_sigma(sigma2, lmin, lmax, t);
    if (theta) *theta = th;
    *n_accepted = 0;
    if (S->m_off > 0) {
        unsigned long long *hm = maxslot(ctx, 3);
        memset_d(ctx, hm, 0, sizeof(unsigned long long));
        max_abs_bits(ctx, prec, S->m_off, heat, hm);
        unsigned long long b = 0;
        d2h(ctx, &b, hm, sizeof(b));
        *n_accepted = filter_similar(ctx, S, heat, prec, th * bits_to_double(b), cap, accepted);
        ctx->sync();
    }
    API_END
}

// ---------------------------------------------------------------- densify / solve

grass_status grass_densify(grass_ctx_t ctx, grass_tree_t T, const grass_params_t *P,
                           const double *h0, const double *v0, grass_sparsifier_t *out,
                           grass_sparsify_stats_t *stats) {
    if (!ctx || !T || !P || !out) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    *out = nullptr;
    need(T->g.nseg == 1, "a batch of graphs: use grass_densify_batch");
    need(h0 && v0, "null h0 / v0");
    need(P->sigma2 > 0, "sigma2 must be > 0");
    need(r_supported(P->r), "r must be 1, 2, 4, 8, 16, 24 or 32");
    need(P->t >= 1, "t must be >= 1");
    need(P->max_rounds >= 1 && P->max_rounds <= GRASS_MAX_ROUNDS, "max_rounds out of range");
    need(P->lmax_iters >= 0, "lmax_iters must be >= 0");
    need(P->inner_maxit >= 0, "inner_maxit must be >= 0");
    need_prec(P->embed_prec);
    const double t0 = now_ms();
    grass_sparsify_stats_t st;
    std::memset(&st, 0, sizeof(st));
    const int64_t n = T->g.n;
    const int r = P->r;
    clear_timeout(ctx);
    memset_d(ctx, ctx->scal.p + DS_RED + DS_ITER, 0, sizeof(double));
    grass_sparsifier_t S = new_sparsifier(ctx, T);
    try {
        void *heat = ctx->scr<char>(SCR_HEAT, (T->g.m + 1) * esize(P->embed_prec));
        int64_t *acc = ctx->scr<int64_t>(SCR_PCG_E, T->g.m + 1);
        // the last lambda_max estimate whose inner solves all converged;
        // round 1's are direct tree solves, so it is set in round 1
        double lmax_trusted = 0.0;
        for (int k = 0; k < P->max_rounds; ++k) {
            double ta = now_ms();
            double lmin = 0.0;
            lambda_min(ctx, S, &lmin);
            int64_t inner = 0;
            memset_d(ctx, ctx->scal.p + DS_RED + DS_CAPPED, 0, sizeof(double));
            // an estimate with a capped solve can neither stop the loop nor
            // set theta_sigma (below), so its power steps end at that solve
            double lmax = lambda_max_impl(ctx, S, v0 + (int64_t)k * n, P->lmax_iters,
                                          P->embed_prec, P->inner_tol, P->inner_maxit, &inner,
                                          true);
            double capped = 0.0;
            d2h(ctx, &capped, ctx->scal.p + DS_RED + DS_CAPPED, sizeof(double));
            st.lmin_est[k] = lmin;
            st.lmax_est[k] = lmax;
            st.lmax_capped[k] = (int64_t)capped;
            double tb = now_ms();
            st.ms_estimate += tb - ta;
            // step 3: a Rayleigh quotient only bounds lambda_max from below,
            // and one taken after inexact inner solves can fall far below it;
            // the stop test trusts an estimate whose inner solves all met
            // inner_tol before inner_maxit
            if (capped == 0.0 && lmax / lmin <= P->sigma2) {
                st.stopped_similar = 1;
                st.inner_iters += inner;
                break;
            }
            // an untrusted estimate does not set theta_sigma either: adding
            // edges to S only lowers lambda_max(L_S^+ L_G), so the last
            // trusted estimate is the best upper value at hand (a capped
            // one can make theta_sigma > 1 and reject every edge)
            if (capped == 0.0 || lmax_trusted == 0.0) lmax_trusted = lmax;
            int64_t moff = S->m_off;
            EmbedOut eo = embed_impl(ctx, S, h0 + (int64_t)k * n * r, r, P->t, P->embed_prec,
                                     P->inner_tol, P->inner_maxit, nullptr, heat);
            inner += eo.inner;
            st.inner_iters += inner;
            double tc = now_ms();
            st.ms_embed += tc - tb;
            st.ms_embed_round[k] = tc - tb;
            double th = theta_sigma(P->sigma2, lmin, lmax_trusted, P->t);
            st.theta[k] = th;
            st.heat_max[k] = eo.heat_max;
            st.embedded_round[k] = moff;
            st.offtree_embedded += moff;
            int64_t na = ctx->similarity_check
                             ? filter_similar(ctx, S, heat, P->embed_prec, th * eo.heat_max,
                                              P->max_add_per_round, acc)
                             : filter_heat(ctx, S, heat, P->embed_prec, th * eo.heat_max,
                                           P->max_add_per_round, acc);
            double td = now_ms();
            st.ms_filter += td - tc;
            st.rounds = k + 1;
            st.added_round[k] = na;
            st.added += na;
            if (na == 0) break;
            sparsifier_add(ctx, S, acc, na);
            ctx->sync();
            st.ms_update += now_ms() - td;
        }
        double iters = 0.0;
        d2h(ctx, &iters, ctx->scal.p + DS_RED + DS_ITER, sizeof(double));
        st.inner_iters += (int64_t)iters;
        ctx->sync();
    } catch (...) {
        delete S;
        throw;
    }
    try {
        check_timeout(ctx);
    } catch (...) {
        delete S;
        throw;
    }
    st.ms_total = now_ms() - t0;
    if (stats) *stats = st;
    *out = S;
    API_END
}

grass_status grass_pcg_solve(grass_ctx_t ctx, grass_sparsifier_t S, const double *b, double *x,
                             double tol, int maxit, grass_prec prec, double refine_tol,
                             double inner_tol, int inner_maxit, grass_solve_stats_t *stats) {
    if (!ctx || !S) return GRASS_ERR_INVALID;
    API_BEGIN(ctx)
    need(S->tree->g.nseg == 1, "a batch of graphs: use grass_pcg_solve_batch");
    need(b && x, "null b / x");
    need(tol > 0 && maxit >= 0, "tol must be > 0, maxit >= 0");
    need_prec(prec);
    need(prec == GRASS_FP64 || (refine_tol > 0 && refine_tol < 1), "refine_tol must be in (0, 1)");
    need(inner_maxit >= 0, "inner_maxit must be >= 0");
    ensure_sdd(ctx, S->tree);
    double t0 = now_ms();
    grass_solve_stats_t st;
    std::memset(&st, 0, sizeof(st));
    try {
        clear_timeout(ctx);
        pcg_solve(ctx, S, b, x, tol, maxit, prec, refine_tol, inner_tol, inner_maxit, &st);
        check_timeout(ctx);
    } catch (const grass::Error &e) {
        st.ms = now_ms() - t0;
        if (stats) *stats = st;
        throw;
    }
    st.ms = now_ms() - t0;
    if (stats) *stats = st;
    API_END
}

}  // extern "C"
