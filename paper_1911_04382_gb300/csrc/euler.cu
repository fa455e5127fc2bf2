// euler.cu -- Euler tour of the spanning tree (forest), built once per tree,
// for the scan form of the grounded tree solve (Sec. III-F: x = L_T^+ b
// grounded at the root; D = 0).
//
// For the tree Laplacian grounded at the root, the current through the edge
// from v up to its parent is the sum of b over v's subtree, and x_v is the
// sum, over the edges on the root path of v, of current / weight.  With the
// vertices laid out along an Euler tour (v's subtree is the stretch between
// the tour's entry into v and its exit from v) both sums are differences of
// prefix sums: two scans replace the leaf-to-root and root-to-leaf sweeps.
//
// Tour: every tree edge gives two directed slots (the adjacency slots of
// its two ends); the slot after (u -> v) is the one after (v -> u) in v's
// slot list, cyclically; each tree's circuit starts at the first slot of its
// root and is cut where it returns to the root.  Positions come from list
// ranking by pointer jumping (distance to the end of the circuit).  The
// preorder numbering (each tree's root, then its vertices in the order the
// tour enters them) and the tour's arrays in that numbering serve solvers
// that keep their vectors in preorder.
#include "common.cuh"

namespace grass {
namespace {

__global__ void k_u8_to_i64(int64_t m, const uint8_t *a, int64_t *b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) b[i] = a[i];
}

__global__ void k_eu_owner(int64_t n, const int32_t *tptr, int32_t *owner) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    for (int32_t s = tptr[v]; s < tptr[v + 1]; ++s) owner[s] = (int32_t)v;
}

// es[2e + side] = the slot of edge e owned by its smaller (side 0) or larger
// (side 1) end
__global__ void k_eu_edgeslots(int64_t L, const int32_t *owner, const int32_t *tocc,
                               const int32_t *tsrc, int32_t *es, const int32_t *eidx) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= L) return;
    const int32_t u = owner[s], v = tocc[s], e = tsrc[s];
    es[2 * (int64_t)eidx[e] + (u < v ? 0 : 1)] = (int32_t)s;
}

// dense index of every tree edge id (in_tree prefix positions)
__global__ void k_eu_tidx(int64_t m, const uint8_t *in_tree, const int64_t *pos, int32_t *eidx) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m && in_tree[e]) eidx[e] = (int32_t)pos[e];
}

__global__ void k_eu_succ(int64_t L, const int32_t *owner, const int32_t *tptr, const int32_t *tocc,
                          const int32_t *tsrc, const int32_t *eidx, const int32_t *es,
                          const uint8_t *isroot, int32_t *succ, int32_t *dist) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= L) return;
    const int32_t u = owner[s], v = tocc[s];
    const int32_t rev = es[2 * (int64_t)eidx[tsrc[s]] + (u < v ? 1 : 0)];   // (v -> u)
    int32_t nx;
    if (rev + 1 < tptr[v + 1]) {
        nx = rev + 1;
    } else {
        nx = isroot[v] ? -1 : tptr[v];   // back at the root after its last slot: the end
    }
    succ[s] = nx;
    dist[s] = nx < 0 ? 0 : 1;
}

// one round of pointer jumping: dist += dist[next], next = next[next]
__global__ void k_eu_jump(int64_t L, const int32_t *nx_in, const int32_t *d_in, int32_t *nx_out,
                          int32_t *d_out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= L) return;
    const int32_t nx = nx_in[s];
    if (nx < 0) {
        nx_out[s] = -1;
        d_out[s] = d_in[s];
    } else {
        nx_out[s] = nx_in[nx];
        d_out[s] = d_in[s] + d_in[nx];
    }
}

// positions of the two slots of every tree edge; the earlier one enters the
// child, the later one leaves it
__global__ void k_eu_final(int64_t mt, const int32_t *es, const int32_t *owner, const int32_t *tocc,
                           const int32_t *tsrc, const int32_t *dist, const int32_t *seg_of,
                           const int64_t *voff, const double *ew, int32_t *tour, int32_t *ein,
                           int32_t *eout, double *pw) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= mt) return;
    const int32_t s0 = es[2 * t], s1 = es[2 * t + 1];
    const int32_t u = owner[s0], v = tocc[s0];
    // tree k's circuit occupies [2 (voff[k] - k), + 2 (n_k - 1)); position =
    // base + length - 1 - distance to the end
    int64_t base = 0, len = 0;
    if (seg_of) {
        const int32_t k = seg_of[u];
        base = 2 * (voff[k] - k);
        len = 2 * (voff[k + 1] - voff[k] - 1);
    } else {
        len = 2 * (int64_t)mt;
    }
    const int64_t p0 = base + len - 1 - dist[s0], p1 = base + len - 1 - dist[s1];
    const int32_t child = p0 < p1 ? v : u;
    const int64_t pin = p0 < p1 ? p0 : p1, pout = p0 < p1 ? p1 : p0;
    ein[child] = (int32_t)pin;
    eout[child] = (int32_t)pout;
    tour[pin] = child;
    tour[pout] = -(child + 1);
    pw[child] = ew[tsrc[s0]];
}

// roots have no entry; every tree's tour starts at 2 (voff[k] - k) (0 for
// a single tree): a head of the segmented scans
__global__ void k_eu_inv(int64_t n, const double *pw, double *ipw, float *ipw32) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const double r = 1.0 / pw[v];
    ipw[v] = r;
    ipw32[v] = (float)r;
}

__global__ void k_eu_roots(int64_t nr, const int32_t *roots, const int64_t *voff, int32_t *ein,
                           int32_t *eout, double *pw, uint8_t *head) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nr) return;
    ein[roots[q]] = -1;
    eout[roots[q]] = -1;
    pw[roots[q]] = 1.0;
    head[voff ? 2 * (voff[q] - q) : 0] = 1;
}

// ---- preorder numbering
__global__ void k_eu_isentry(int64_t L, const int32_t *tour, int64_t *f) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < L) f[p] = tour[p] >= 0 ? 1 : 0;
}

// pre[v]: a root takes its tree's first slot (the tree's vertex offset); a
// vertex entered at position p takes (entries before p) + (trees up to and
// including its own), i.e. one slot after its tree's root and the vertices
// entered before it
__global__ void k_eu_pre(int64_t n, const int32_t *ein, const int64_t *epos, const int32_t *seg_of,
                         const int64_t *voff, int32_t *pre, int32_t *vert) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int64_t t = seg_of ? seg_of[v] : 0;
    const int64_t k = ein[v] >= 0 ? epos[ein[v]] + t + 1 : (voff ? voff[t] : 0);
    pre[v] = (int32_t)k;
    vert[k] = (int32_t)v;
}

__global__ void k_eu_tourpre(int64_t L, const int32_t *tour, const int32_t *pre, int32_t *out) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L) return;
    const int32_t t = tour[p];
    out[p] = t >= 0 ? pre[t] : -(pre[-t - 1] + 1);
}

// every tree's root slot in the preorder (the tree's vertex offset)
__global__ void k_eu_headpre(int64_t nr, const int64_t *voff, uint8_t *head_pre) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nr) head_pre[voff ? voff[q] : 0] = 1;
}

__global__ void k_eu_prevals(int64_t n, const int32_t *vert, const int32_t *ein, const int32_t *eout,
                             const double *ipw, const float *ipw32, int32_t *ein_p, int32_t *eout_p,
                             double *ipw_p, float *ipw32_p) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t v = vert[k];
    ein_p[k] = ein[v];
    eout_p[k] = eout[v];
    ipw_p[k] = ipw[v];
    ipw32_p[k] = ipw32[v];
}

}  // namespace

void euler_build(grass_ctx_t ctx, grass_tree_t T, const int32_t *tptr, const int32_t *tocc,
                 const int32_t *tsrc, int64_t L) {
    const GraphData &g = T->g;
    const int64_t n = g.n, m = g.m, mt = L / 2;
    EulerTour &E = T->euler;
    DBuf<int32_t> owner, es, eidx, nx0, nx1, d0, d1;
    DBuf<int64_t> flag, pos;
    owner.alloc(L);
    es.alloc(L);
    eidx.alloc(m);
    launch(ctx, k_eu_owner, cdiv(n, kBlock), kBlock, 0, n, tptr, owner.p);
    // dense tree-edge index: prefix positions of in_tree
    flag.alloc(m + 1);
    pos.alloc(m + 1);
    launch(ctx, k_u8_to_i64, cdiv(m, kBlock), kBlock, 0, m, (const uint8_t *)T->in_tree.p, flag.p);
    int64_t cnt = 0;
    scan_i64(ctx, flag.p, pos.p, m, &cnt);
    if (cnt != mt) fail(GRASS_ERR_CUDA, "Euler tour: tree edge count mismatch");
    launch(ctx, k_eu_tidx, cdiv(m, kBlock), kBlock, 0, m, (const uint8_t *)T->in_tree.p,
           (const int64_t *)pos.p, eidx.p);
    launch(ctx, k_eu_edgeslots, cdiv(L, kBlock), kBlock, 0, L, (const int32_t *)owner.p, tocc, tsrc,
           es.p, (const int32_t *)eidx.p);
    nx0.alloc(L);
    nx1.alloc(L);
    d0.alloc(L);
    d1.alloc(L);
    launch(ctx, k_eu_succ, cdiv(L, kBlock), kBlock, 0, L, (const int32_t *)owner.p, tptr, tocc, tsrc,
           (const int32_t *)eidx.p, (const int32_t *)es.p, (const uint8_t *)T->isroot.p, nx0.p,
           d0.p);
    int rounds = 1;
    while ((int64_t(1) << rounds) < L) ++rounds;
    for (int k = 0; k <= rounds; ++k) {
        launch(ctx, k_eu_jump, cdiv(L, kBlock), kBlock, 0, L, (const int32_t *)nx0.p,
               (const int32_t *)d0.p, nx1.p, d1.p);
        std::swap(nx0.p, nx1.p);
        std::swap(d0.p, d1.p);
    }
    E.L = L;
    E.tour.alloc(L);
    E.ein.alloc(n);
    E.eout.alloc(n);
    E.pw.alloc(n);
    launch(ctx, k_eu_final, cdiv(mt, kBlock), kBlock, 0, mt, (const int32_t *)es.p,
           (const int32_t *)owner.p, tocc, tsrc, (const int32_t *)d0.p,
           g.nseg > 1 ? (const int32_t *)g.seg_of.p : nullptr,
           g.nseg > 1 ? (const int64_t *)g.seg_voff_d.p : nullptr, (const double *)g.ew64.p,
           E.tour.p, E.ein.p, E.eout.p, E.pw.p);
    E.head.alloc(L);
    memset_d(ctx, E.head.p, 0, L);
    launch(ctx, k_eu_roots, cdiv(T->nroots, kBlock), kBlock, 0, T->nroots,
           (const int32_t *)T->roots.p, g.nseg > 1 ? (const int64_t *)g.seg_voff_d.p : nullptr,
           E.ein.p, E.eout.p, E.pw.p, E.head.p);
    E.ipw.alloc(n);
    E.ipw32.alloc(n);
    launch(ctx, k_eu_inv, cdiv(n, kBlock), kBlock, 0, n, (const double *)E.pw.p, E.ipw.p, E.ipw32.p);
    // preorder numbering and the tour / per-vertex arrays in it
    {
        DBuf<int64_t> ent, epos;
        ent.alloc(L + 1);
        epos.alloc(L + 1);
        launch(ctx, k_eu_isentry, cdiv(L, kBlock), kBlock, 0, L, (const int32_t *)E.tour.p, ent.p);
        int64_t ne = 0;
        scan_i64(ctx, ent.p, epos.p, L, &ne);
        if (ne != n - T->nroots) fail(GRASS_ERR_CUDA, "Euler tour: entry count mismatch");
        E.pre.alloc(n);
        E.vert.alloc(n);
        launch(ctx, k_eu_pre, cdiv(n, kBlock), kBlock, 0, n, (const int32_t *)E.ein.p,
               (const int64_t *)epos.p, g.nseg > 1 ? (const int32_t *)g.seg_of.p : nullptr,
               g.nseg > 1 ? (const int64_t *)g.seg_voff_d.p : nullptr, E.pre.p, E.vert.p);
        E.tour_pre.alloc(L);
        launch(ctx, k_eu_tourpre, cdiv(L, kBlock), kBlock, 0, L, (const int32_t *)E.tour.p,
               (const int32_t *)E.pre.p, E.tour_pre.p);
        E.head_pre.alloc(n);
        memset_d(ctx, E.head_pre.p, 0, n);
        launch(ctx, k_eu_headpre, cdiv(T->nroots, kBlock), kBlock, 0, T->nroots,
               g.nseg > 1 ? (const int64_t *)g.seg_voff_d.p : nullptr, E.head_pre.p);
        E.ein_pre.alloc(n);
        E.eout_pre.alloc(n);
        E.ipw_pre.alloc(n);
        E.ipw32_pre.alloc(n);
        launch(ctx, k_eu_prevals, cdiv(n, kBlock), kBlock, 0, n, (const int32_t *)E.vert.p,
               (const int32_t *)E.ein.p, (const int32_t *)E.eout.p, (const double *)E.ipw.p,
               (const float *)E.ipw32.p, E.ein_pre.p, E.eout_pre.p, E.ipw_pre.p, E.ipw32_pre.p);
    }
    E.built = true;
}

}  // namespace grass
