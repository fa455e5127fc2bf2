// mst.cu -- maximum-weight spanning tree by Boruvka rounds.
//
// Edges are compared by the strict total order (w descending, edge id
// ascending), so the maximum spanning tree is unique and Boruvka's
// per-component choices agree exactly with Kruskal's greedy order.  The
// comparison is exact: positive doubles order like their bit patterns, so
// the heaviest incident weight is an integer atomicMax and the tie on equal
// weight an atomicMin on the edge id.
#include "common.cuh"

namespace grass {

constexpr int32_t kNoEdge = 0x7F7F7F7F;   // byte-wise memset value 0x7F

__device__ inline unsigned long long wbits(double w) { return (unsigned long long)__double_as_longlong(w); }

__global__ void k_bor_init(int64_t n, int32_t *comp) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) comp[v] = (int32_t)v;
}

__global__ void k_iota(int64_t m, int32_t *a) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) a[i] = (int32_t)i;
}

__global__ void k_bor_max(int64_t na, const int32_t *act, const int32_t *eu, const int32_t *ev,
                          const double *ew, const int32_t *comp, unsigned long long *bw) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= na) return;
    int32_t e = act[i];
    int32_t cu = comp[eu[e]], cv = comp[ev[e]];
    if (cu == cv) return;
    unsigned long long b = wbits(ew[e]);
    atomicMax(bw + cu, b);
    atomicMax(bw + cv, b);
}

__global__ void k_bor_min(int64_t na, const int32_t *act, const int32_t *eu, const int32_t *ev,
                          const double *ew, const int32_t *comp, const unsigned long long *bw,
                          int32_t *be) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= na) return;
    int32_t e = act[i];
    int32_t cu = comp[eu[e]], cv = comp[ev[e]];
    if (cu == cv) return;
    unsigned long long b = wbits(ew[e]);
    if (b == bw[cu]) atomicMin(be + cu, e);
    if (b == bw[cv]) atomicMin(be + cv, e);
}

// hook[c] = component across c's best edge (roots only).
__global__ void k_bor_hook(int64_t n, const int32_t *comp, const int32_t *be, const int32_t *eu,
                           const int32_t *ev, int32_t *hook) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || comp[c] != c) return;
    int32_t e = be[c];
    if (e == kNoEdge) {
        hook[c] = (int32_t)c;
        return;
    }
    int32_t a = comp[eu[e]], b = comp[ev[e]];
    hook[c] = a == c ? b : a;
}

// A pair of components that chose the same edge points at each other; the
// smaller id stays a root.  Every component that still hooks adds its edge.
__global__ void k_bor_break(int64_t n, const int32_t *comp, const int32_t *hook, const int32_t *be,
                            int32_t *nh, uint8_t *in_tree, unsigned int *nhooked) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || comp[c] != c) return;
    int32_t h = hook[c];
    int32_t r = h;
    if (h != c && hook[h] == c && c < h) r = (int32_t)c;
    nh[c] = r;
    if (r != c) {
        in_tree[be[c]] = 1;
        atomicAdd(nhooked, 1u);
    }
}

__global__ void k_bor_jump(int64_t n, const int32_t *comp, int32_t *nh, int *changed) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || comp[c] != c) return;
    int32_t p = nh[c];
    int32_t pp = nh[p];
    if (p != pp) {
        nh[c] = pp;
        *changed = 1;
    }
}

__global__ void k_bor_relabel(int64_t n, int32_t *comp, const int32_t *nh) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) comp[v] = nh[comp[v]];
}

__global__ void k_bor_flag(int64_t na, const int32_t *act, const int32_t *eu, const int32_t *ev,
                           const int32_t *comp, int64_t *flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= na) return;
    int32_t e = act[i];
    flag[i] = comp[eu[e]] != comp[ev[e]] ? 1 : 0;
}

__global__ void k_bor_compact(int64_t na, const int32_t *act, const int64_t *flag,
                              const int64_t *pos, int32_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= na || !flag[i]) return;
    out[pos[i]] = act[i];
}

void mst_boruvka(grass_ctx_t ctx, const GraphData &g, uint8_t *in_tree) {
    mst_boruvka_w(ctx, g, g.ew64.p, in_tree);
}

// The same over the graph's edges with weights ew (device, m positive
// doubles) in place of the graph's own.
void mst_boruvka_w(grass_ctx_t ctx, const GraphData &g, const double *ew, uint8_t *in_tree) {
    const int64_t n = g.n, m = g.m;
    DBuf<int32_t> comp, hook, nh, be, act0, act1;
    DBuf<unsigned long long> bw;
    DBuf<int64_t> flag, pos;
    comp.alloc(n);
    hook.alloc(n);
    nh.alloc(n);
    be.alloc(n);
    bw.alloc(n);
    act0.alloc(m);
    act1.alloc(m);
    flag.alloc(m + 1);
    pos.alloc(m + 1);
    unsigned int *nhooked = (unsigned int *)(ctx->flags.p + 1);
    int *changed = ctx->flags.p + 2;
    memset_d(ctx, in_tree, 0, (size_t)m);
    launch(ctx, k_bor_init, cdiv(n, kBlock), kBlock, 0, n, comp.p);
    launch(ctx, k_iota, cdiv(m, kBlock), kBlock, 0, m, act0.p);
    int32_t *act = act0.p, *act_next = act1.p;
    int64_t na = m, roots = n;
    for (int round = 0; roots > g.nseg; ++round) {
        if (round > 64) fail(GRASS_ERR_CUDA, "Boruvka did not converge");
        memset_d(ctx, bw.p, 0, n * sizeof(unsigned long long));
        memset_d(ctx, be.p, 0x7F, n * sizeof(int32_t));     // kNoEdge
        launch(ctx, k_bor_max, cdiv(na, kBlock), kBlock, 0, na, (const int32_t *)act, g.eu.p,
               g.ev.p, ew, (const int32_t *)comp.p, bw.p);
        launch(ctx, k_bor_min, cdiv(na, kBlock), kBlock, 0, na, (const int32_t *)act, g.eu.p,
               g.ev.p, ew, (const int32_t *)comp.p, (const unsigned long long *)bw.p, be.p);
        launch(ctx, k_bor_hook, cdiv(n, kBlock), kBlock, 0, n, (const int32_t *)comp.p,
               (const int32_t *)be.p, g.eu.p, g.ev.p, hook.p);
        memset_d(ctx, nhooked, 0, sizeof(unsigned int));
        launch(ctx, k_bor_break, cdiv(n, kBlock), kBlock, 0, n, (const int32_t *)comp.p,
               (const int32_t *)hook.p, (const int32_t *)be.p, nh.p, in_tree, nhooked);
        for (int j = 0; j < 64; ++j) {
            memset_d(ctx, changed, 0, sizeof(int));
            launch(ctx, k_bor_jump, cdiv(n, kBlock), kBlock, 0, n, (const int32_t *)comp.p, nh.p,
                   changed);
            launch(ctx, k_bor_jump, cdiv(n, kBlock), kBlock, 0, n, (const int32_t *)comp.p, nh.p,
                   changed);
            int ch = 0;
            d2h(ctx, &ch, changed, sizeof(int));
            if (!ch) break;
        }
        launch(ctx, k_bor_relabel, cdiv(n, kBlock), kBlock, 0, n, comp.p, (const int32_t *)nh.p);
        unsigned int hooked = 0;
        d2h(ctx, &hooked, nhooked, sizeof(unsigned int));
        if (hooked == 0) {
            fail(GRASS_ERR_DISCONNECTED,
                 g.nseg > 1 ? "the batch has " + std::to_string(roots) + " connected components for " +
                                  std::to_string(g.nseg) + " graphs"
                            : "graph has " + std::to_string(roots) + " connected components");
        }
        roots -= hooked;
        if (roots <= g.nseg) break;
        launch(ctx, k_bor_flag, cdiv(na, kBlock), kBlock, 0, na, (const int32_t *)act, g.eu.p,
               g.ev.p, (const int32_t *)comp.p, flag.p);
        int64_t kept = 0;
        scan_i64(ctx, flag.p, pos.p, na, &kept);
        launch(ctx, k_bor_compact, cdiv(na, kBlock), kBlock, 0, na, (const int32_t *)act,
               (const int64_t *)flag.p, (const int64_t *)pos.p, act_next);
        std::swap(act, act_next);
        na = kept;
    }
}

}  // namespace grass
