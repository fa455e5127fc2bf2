// lsst.cu -- low-stretch spanning tree and per-edge stretch.
//
// The paper's backbone is a low-stretch spanning tree (Sec. III-B); its
// total stretch st_T(G) = sum_e w_e R_T(e) is Tr(L_T^+ L_G), the quantity
// the sparsifier's condition number starts from.  The construction here is
// the classic clustering one (Alon, Karp, Peleg and West) with shifted
// low-diameter decompositions (Miller, Peng and Xu), in a deterministic form
// that a CPU restatement reproduces bit for bit:
//
//   * class of edge e = emax - e_e, e_e the binary exponent of w_e (frexp),
//     so class 0 holds the heaviest binade;
//   * for each class c and level = 0, 1, ...: the active edges are those of
//     classes <= c whose endpoints lie in different clusters (a cluster is
//     named by a vertex id; every vertex starts alone); none left ends the
//     class;
//   * every cluster x on an active edge draws shift(x) = 3 * min(20, leading
//     zeros of SplitMix64(seed + (x+1) G + (1000003 c + level) H)) and starts
//     at round S - shift(x), S the largest shift of the level;
//   * round t: an unclaimed cluster next to clusters claimed in round t-1
//     joins the centre with the smallest (start, centre id) among theirs,
//     through the heaviest edge (smallest id on equal weight) to such a
//     neighbour, and that edge joins the tree; then every unclaimed cluster
//     whose start is t becomes a centre.  Every cluster is claimed by round S;
//   * the clusters are renamed by their centres.
//
// The three-key choice is three passes of integer atomics: the smallest
// (start << 32 | centre), then the largest weight bit pattern among the
// edges carrying that key (positive doubles order like their bits), then
// the smallest edge id among those.
//
// Stretch: parents from the Euler tour's entry order, path resistances to
// the root and the ancestor table by pointer doubling (sums of positive
// terms only), and each edge's lowest common ancestor by binary lifting.
#include "common.cuh"
#include "tree_solve.cuh"

namespace grass {

namespace {

constexpr unsigned long long kNoKey = ~0ull;
constexpr int32_t kNoEdgeId = 0x7FFFFFFF;
constexpr unsigned long long kGolden = 0x9E3779B97F4A7C15ull;
constexpr unsigned long long kLevelMul = 0xD1B54A32D192ED03ull;
constexpr int kShiftScale = 3;
constexpr int kShiftCap = 20;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + kGolden;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int ls_shift(unsigned long long seed, int cls, int level, int32_t x) {
    unsigned long long st = seed + (unsigned long long)(x + 1) * kGolden +
                            ((unsigned long long)cls * 1000003ull + (unsigned long long)level) * kLevelMul;
    int lz = __clzll((long long)splitmix64(st));
    return kShiftScale * (lz < kShiftCap ? lz : kShiftCap);
}

__device__ __forceinline__ unsigned long long wbits(double w) {
    return (unsigned long long)__double_as_longlong(w);
}

__global__ void k_ls_exp(int64_t m, const double *ew, int32_t *ex, int *emax) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int v = INT_MIN;
    if (e < m) {
        int x;
        frexp(ew[e], &x);
        ex[e] = x;
        v = x;
    }
    for (int d = 16; d > 0; d >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, d));
    if ((threadIdx.x & 31) == 0 && v != INT_MIN) atomicMax(emax, v);
}

__global__ void k_ls_cls(int64_t m, const int *emax, int32_t *ex, int *cmax) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int v = 0;
    if (e < m) {
        v = *emax - ex[e];
        ex[e] = v;
    }
    for (int d = 16; d > 0; d >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, d));
    if ((threadIdx.x & 31) == 0) atomicMax(cmax, v);
}

__global__ void k_ls_present(int64_t m, const int32_t *cls, uint8_t *present) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) present[cls[e]] = 1;
}

__global__ void k_ls_iota(int64_t n, int32_t *a, int32_t *b) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) {
        a[v] = (int32_t)v;
        b[v] = (int32_t)v;
    }
}

// flag[e] = 1 for the edges of classes <= c between different clusters
__global__ void k_ls_cflag(int64_t m, int c, const int32_t *cls, const int32_t *eu,
                           const int32_t *ev, const int32_t *label, int64_t *flag) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    flag[e] = (cls[e] <= c && label[eu[e]] != label[ev[e]]) ? 1 : 0;
}

__global__ void k_ls_cfill(int64_t m, const int64_t *flag, const int64_t *pos, const int32_t *eu,
                           const int32_t *ev, const int32_t *label, int32_t *act, int32_t *ca,
                           int32_t *cb) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m || !flag[e]) return;
    int64_t k = pos[e];
    act[k] = (int32_t)e;
    ca[k] = label[eu[e]];
    cb[k] = label[ev[e]];
}

// The level's clusters: each cluster on an active edge is listed once (the
// first writer of this level's stamp appends it); S = the largest shift.
__global__ void k_ls_xmark(int64_t na, const int32_t *ca, const int32_t *cb, int32_t stamp,
                           int32_t *mark, int32_t *xl, unsigned int *nx, int *smax,
                           unsigned long long seed, int cls, int level) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    int32_t e2[2] = {ca[k], cb[k]};
    for (int s = 0; s < 2; ++s) {
        int32_t x = e2[s];
        if (atomicExch(mark + x, stamp) != stamp) {
            unsigned int i = atomicAdd(nx, 1u);
            xl[i] = x;
            atomicMax(smax, ls_shift(seed, cls, level, x));
        }
    }
}

__global__ void k_ls_xinit(int64_t nx, const int32_t *xl, const int *smax, unsigned long long seed,
                           int cls, int level, int32_t *ctr, int32_t *when, int32_t *start,
                           unsigned long long *key, unsigned long long *wb, int32_t *eb) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    int32_t x = xl[i];
    ctr[x] = -1;
    when[x] = -1;
    start[x] = *smax - ls_shift(seed, cls, level, x);
    key[x] = kNoKey;
    wb[x] = 0ull;
    eb[x] = kNoEdgeId;
}

__device__ __forceinline__ unsigned long long ls_key(const int32_t *start, int32_t c) {
    return ((unsigned long long)(uint32_t)start[c] << 32) | (uint32_t)c;
}

// Pass 1: smallest (start, centre) offered to each unclaimed cluster by its
// neighbours claimed in round t - 1.
__global__ void k_ls_offer(int64_t na, const int32_t *ca, const int32_t *cb, const int32_t *ctr,
                           const int32_t *when, const int32_t *start, int t,
                           unsigned long long *key) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    int32_t x = ca[k], y = cb[k];
    int32_t cx = ctr[x], cy = ctr[y];
    if (cx < 0 && cy >= 0 && when[y] == t - 1) atomicMin(key + x, ls_key(start, cy));
    else if (cy < 0 && cx >= 0 && when[x] == t - 1) atomicMin(key + y, ls_key(start, cx));
}

// Pass 2: heaviest edge carrying the winning offer.
__global__ void k_ls_heavy(int64_t na, const int32_t *act, const int32_t *ca, const int32_t *cb,
                           const int32_t *ctr, const int32_t *when, const int32_t *start, int t,
                           const unsigned long long *key, const double *ew,
                           unsigned long long *wb) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    int32_t x = ca[k], y = cb[k];
    int32_t cx = ctr[x], cy = ctr[y];
    if (cx < 0 && cy >= 0 && when[y] == t - 1) {
        if (ls_key(start, cy) == key[x]) atomicMax(wb + x, wbits(ew[act[k]]));
    } else if (cy < 0 && cx >= 0 && when[x] == t - 1) {
        if (ls_key(start, cx) == key[y]) atomicMax(wb + y, wbits(ew[act[k]]));
    }
}

// Pass 3: smallest id among those heaviest edges.
__global__ void k_ls_eid(int64_t na, const int32_t *act, const int32_t *ca, const int32_t *cb,
                         const int32_t *ctr, const int32_t *when, const int32_t *start, int t,
                         const unsigned long long *key, const double *ew,
                         const unsigned long long *wb, int32_t *eb) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    int32_t x = ca[k], y = cb[k];
    int32_t cx = ctr[x], cy = ctr[y];
    int32_t e = act[k];
    if (cx < 0 && cy >= 0 && when[y] == t - 1) {
        if (ls_key(start, cy) == key[x] && wbits(ew[e]) == wb[x]) atomicMin(eb + x, e);
    } else if (cy < 0 && cx >= 0 && when[x] == t - 1) {
        if (ls_key(start, cx) == key[y] && wbits(ew[e]) == wb[y]) atomicMin(eb + y, e);
    }
}

// Commit round t: joins first, then the new centres.
__global__ void k_ls_commit(int64_t nx, const int32_t *xl, int t, const unsigned long long *key,
                            const int32_t *eb, const int32_t *start, int32_t *ctr, int32_t *when,
                            uint8_t *in_tree) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    int32_t x = xl[i];
    if (ctr[x] >= 0) return;
    unsigned long long kk = key[x];
    if (kk != kNoKey) {
        ctr[x] = (int32_t)(uint32_t)(kk & 0xFFFFFFFFull);
        when[x] = t;
        const int32_t e = eb[x];
        if (e != kNoEdgeId) in_tree[e] = 1;
    } else if (start[x] == t) {
        ctr[x] = x;
        when[x] = t;
    }
}

// The four passes of round t over items i0, i0 + st, ... (one block's
// threads, or the grid's).
__device__ __forceinline__ void ls_pass_offer(int64_t na, const int32_t *ca, const int32_t *cb,
                                              const int32_t *ctr, const int32_t *when,
                                              const int32_t *start, int t, unsigned long long *key,
                                              int64_t i0, int64_t st) {
    for (int64_t k = i0; k < na; k += st) {
        const int32_t x = ca[k], y = cb[k];
        const int32_t cx = ctr[x], cy = ctr[y];
        if (cx < 0 && cy >= 0 && when[y] == t - 1) atomicMin(key + x, ls_key(start, cy));
        else if (cy < 0 && cx >= 0 && when[x] == t - 1) atomicMin(key + y, ls_key(start, cx));
    }
}

__device__ __forceinline__ void ls_pass_heavy(int64_t na, const int32_t *act, const int32_t *ca,
                                              const int32_t *cb, const int32_t *ctr,
                                              const int32_t *when, const int32_t *start, int t,
                                              const unsigned long long *key, const double *ew,
                                              unsigned long long *wb, int64_t i0, int64_t st) {
    for (int64_t k = i0; k < na; k += st) {
        const int32_t x = ca[k], y = cb[k];
        const int32_t cx = ctr[x], cy = ctr[y];
        if (cx < 0 && cy >= 0 && when[y] == t - 1) {
            if (ls_key(start, cy) == key[x]) atomicMax(wb + x, wbits(ew[act[k]]));
        } else if (cy < 0 && cx >= 0 && when[x] == t - 1) {
            if (ls_key(start, cx) == key[y]) atomicMax(wb + y, wbits(ew[act[k]]));
        }
    }
}

__device__ __forceinline__ void ls_pass_eid(int64_t na, const int32_t *act, const int32_t *ca,
                                            const int32_t *cb, const int32_t *ctr,
                                            const int32_t *when, const int32_t *start, int t,
                                            const unsigned long long *key, const double *ew,
                                            const unsigned long long *wb, int32_t *eb, int64_t i0,
                                            int64_t st) {
    for (int64_t k = i0; k < na; k += st) {
        const int32_t x = ca[k], y = cb[k];
        const int32_t cx = ctr[x], cy = ctr[y];
        const int32_t e = act[k];
        if (cx < 0 && cy >= 0 && when[y] == t - 1) {
            if (ls_key(start, cy) == key[x] && wbits(ew[e]) == wb[x]) atomicMin(eb + x, e);
        } else if (cy < 0 && cx >= 0 && when[x] == t - 1) {
            if (ls_key(start, cx) == key[y] && wbits(ew[e]) == wb[y]) atomicMin(eb + y, e);
        }
    }
}

__device__ __forceinline__ void ls_pass_commit(int64_t nx, const int32_t *xl, int t,
                                               const unsigned long long *key, const int32_t *eb,
                                               const int32_t *start, int32_t *ctr, int32_t *when,
                                               uint8_t *in_tree, int64_t i0, int64_t st) {
    for (int64_t i = i0; i < nx; i += st) {
        const int32_t x = xl[i];
        if (ctr[x] >= 0) continue;
        const unsigned long long kk = key[x];
        if (kk != kNoKey) {
            ctr[x] = (int32_t)(uint32_t)(kk & 0xFFFFFFFFull);
            when[x] = t;
            const int32_t e = eb[x];
            if (e != kNoEdgeId) in_tree[e] = 1;
        } else if (start[x] == t) {
            ctr[x] = x;
            when[x] = t;
        }
    }
}

// A whole level (rounds 0..S, the same four passes) in one block, for the
// many small levels (at most ctx->lsst_small_level active edges):
// __syncthreads between the passes in place of launches.
constexpr int kLevelBlock = 1024;

__global__ void __launch_bounds__(kLevelBlock) k_ls_level(
    int64_t na, int64_t nx, const int32_t *act, const int32_t *ca, const int32_t *cb,
    const int32_t *xl, const int *smax, const int32_t *start, const double *ew, int32_t *ctr,
    int32_t *when, unsigned long long *key, unsigned long long *wb, int32_t *eb,
    uint8_t *in_tree) {
    const int S = *smax;
    const int64_t i0 = threadIdx.x, st = blockDim.x;
    for (int t = 0; t <= S; ++t) {
        ls_pass_offer(na, ca, cb, ctr, when, start, t, key, i0, st);
        __syncthreads();
        ls_pass_heavy(na, act, ca, cb, ctr, when, start, t, key, ew, wb, i0, st);
        __syncthreads();
        ls_pass_eid(na, act, ca, cb, ctr, when, start, t, key, ew, wb, eb, i0, st);
        __syncthreads();
        ls_pass_commit(nx, xl, t, key, eb, start, ctr, when, in_tree, i0, st);
        __syncthreads();
    }
}

// The larger levels in one cooperative launch per level: the same passes
// over the grid's threads, bounded grid barriers between them in place of
// four launches per round.
__global__ void __launch_bounds__(kLevelBlock) k_ls_level_grid(
    int64_t na, int64_t nx, const int32_t *act, const int32_t *ca, const int32_t *cb,
    const int32_t *xl, const int *smax, const int32_t *start, const double *ew, int32_t *ctr,
    int32_t *when, unsigned long long *key, unsigned long long *wb, int32_t *eb,
    uint8_t *in_tree, unsigned int *bar, long long budget, int *err) {
    const int S = *smax;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    unsigned int epoch = 0;
    for (int t = 0; t <= S; ++t) {
        ls_pass_offer(na, ca, cb, ctr, when, start, t, key, i0, st);
        if (!grid_sync(bar, budget, err, epoch)) return;
        ls_pass_heavy(na, act, ca, cb, ctr, when, start, t, key, ew, wb, i0, st);
        if (!grid_sync(bar, budget, err, epoch)) return;
        ls_pass_eid(na, act, ca, cb, ctr, when, start, t, key, ew, wb, eb, i0, st);
        if (!grid_sync(bar, budget, err, epoch)) return;
        ls_pass_commit(nx, xl, t, key, eb, start, ctr, when, in_tree, i0, st);
        if (!grid_sync(bar, budget, err, epoch)) return;
    }
}

__global__ void k_ls_relabel(int64_t n, const int32_t *ctr, int32_t *label) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t c = ctr[label[v]];
    if (c >= 0) label[v] = c;
}

// Next level's active edges: endpoints renamed by their centres.
__global__ void k_ls_nflag(int64_t na, const int32_t *ca, const int32_t *cb, const int32_t *ctr,
                           int64_t *flag) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    flag[k] = ctr[ca[k]] != ctr[cb[k]] ? 1 : 0;
}

__global__ void k_ls_nfill(int64_t na, const int64_t *flag, const int64_t *pos, const int32_t *act,
                           const int32_t *ca, const int32_t *cb, const int32_t *ctr, int32_t *act2,
                           int32_t *ca2, int32_t *cb2) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na || !flag[k]) return;
    int64_t j = pos[k];
    act2[j] = act[k];
    ca2[j] = ctr[ca[k]];
    cb2[j] = ctr[cb[k]];
}

__global__ void k_ls_count(int64_t m, const uint8_t *in_tree, unsigned long long *cnt) {
    unsigned long long c = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        c += in_tree[e] != 0;
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// ---------------------------------------------------------------- stretch

// parent of the later-entered endpoint of every tree edge, and the edge's
// resistance on that endpoint
__global__ void k_st_parent(int64_t m, const uint8_t *in_tree, const int32_t *eu,
                            const int32_t *ev, const double *ew, const int32_t *ein,
                            int32_t *par, double *res) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m || !in_tree[e]) return;
    int32_t u = eu[e], v = ev[e];
    int32_t child = ein[u] < ein[v] ? v : u;
    int32_t p = child == u ? v : u;
    par[child] = p;
    res[child] = 1.0 / ew[e];
}

__global__ void k_st_rootinit(int64_t n, const uint8_t *isroot, int32_t *par, double *res,
                              int32_t *dep) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    if (isroot[v]) {
        par[v] = (int32_t)v;
        res[v] = 0.0;
        dep[v] = 0;
    } else {
        dep[v] = 1;
    }
}

// one doubling step: the 2^k-th ancestor, and the resistance and depth
// accumulated along the jump (anc_out = anc_in o anc_in)
__global__ void k_st_jump(int64_t n, const int32_t *anc_in, const double *res_in,
                          const int32_t *dep_in, int32_t *anc_out, double *res_out,
                          int32_t *dep_out, int *changed) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t a = anc_in[v];
    int32_t aa = anc_in[a];
    anc_out[v] = aa;
    res_out[v] = res_in[v] + (a != aa ? res_in[a] : 0.0);
    dep_out[v] = dep_in[v] + (a != aa ? dep_in[a] : 0);
    if (a != aa) *changed = 1;
}

// st[e] = w_e (R(u) + R(v) - 2 R(lca)), R = resistance to the root
__global__ void k_st_edge(int64_t m, int K, int64_t n, const int32_t *anc, const int32_t *eu,
                          const int32_t *ev, const double *ew, const double *dist,
                          const int32_t *depth, double *st) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    int32_t a = eu[e], b = ev[e];
    if (depth[a] < depth[b]) {
        int32_t t = a;
        a = b;
        b = t;
    }
    int32_t diff = depth[a] - depth[b];
    for (int k = 0; diff; ++k, diff >>= 1)
        if (diff & 1) a = anc[(int64_t)k * n + a];
    if (a != b) {
        for (int k = K - 1; k >= 0; --k) {
            int32_t pa = anc[(int64_t)k * n + a], pb = anc[(int64_t)k * n + b];
            if (pa != pb) {
                a = pa;
                b = pb;
            }
        }
        a = anc[a];
    }
    st[e] = ew[e] * (dist[eu[e]] + dist[ev[e]] - 2.0 * dist[a]);
}

// deterministic sum: fixed grid, fixed per-thread order, fixed tree
__global__ void k_st_part(int64_t m, const double *x, double *part) {
    __shared__ double sh[kBlock];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        s += x[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int d = kBlock / 2; d > 0; d >>= 1) {
        if ((int)threadIdx.x < d) sh[threadIdx.x] += sh[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_st_final(int nb, const double *part, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += part[i];
        *out = s;
    }
}

}  // namespace

void lsst_build(grass_ctx_t ctx, const GraphData &g, uint64_t seed, uint8_t *in_tree,
                LsstStats *stats) {
    const int64_t n = g.n, m = g.m;
    if (n > 2147483647LL || m > 2147483646LL) fail(GRASS_ERR_INVALID, "graph too large for the low-stretch tree");
    memset_d(ctx, in_tree, 0, (size_t)m);
    DBuf<int32_t> cls, label, ctr, when, start, mark, xl, eb;
    DBuf<unsigned long long> key, wb;
    DBuf<int32_t> act[2], ca[2], cb[2];
    DBuf<int64_t> flag, pos;
    DBuf<int> small;   // [0] emax, [1] class max, [2] S, [3] count x
    cls.alloc(m);
    label.alloc(n);
    ctr.alloc(n);
    when.alloc(n);
    start.alloc(n);
    mark.alloc(n);
    xl.alloc(n);
    eb.alloc(n);
    key.alloc(n);
    wb.alloc(n);
    for (int i = 0; i < 2; ++i) {
        act[i].alloc(m);
        ca[i].alloc(m);
        cb[i].alloc(m);
    }
    flag.alloc(m);
    pos.alloc(m + 1);
    small.alloc(4);

    clear_timeout(ctx);
    const int init_small[4] = {INT_MIN, 0, 0, 0};
    h2d(ctx, small.p, init_small, sizeof(init_small));
    launch(ctx, k_ls_exp, cdiv(m, kBlock), kBlock, 0, m, (const double *)g.ew64.p, cls.p, small.p);
    launch(ctx, k_ls_cls, cdiv(m, kBlock), kBlock, 0, m, (const int *)small.p, cls.p, small.p + 1);
    int hs[4];
    d2h(ctx, hs, small.p, sizeof(hs));
    const int nclass = hs[1] + 1;
    // classes without edges of their own change nothing (the previous class
    // ended with every component of its edges contracted): skipped
    std::vector<uint8_t> present(nclass, 0);
    {
        DBuf<uint8_t> pres;
        pres.alloc(nclass);
        memset_d(ctx, pres.p, 0, nclass);
        launch(ctx, k_ls_present, cdiv(m, kBlock), kBlock, 0, m, (const int32_t *)cls.p, pres.p);
        d2h(ctx, present.data(), pres.p, nclass);
    }
    launch(ctx, k_ls_iota, cdiv(n, kBlock), kBlock, 0, n, label.p, ctr.p);
    memset_d(ctx, mark.p, 0, (size_t)n * sizeof(int32_t));

    int32_t stamp = 0;
    int64_t levels = 0, rounds = 0, edge_passes = 0;
    int cur = 0;
    for (int c = 0; c < nclass; ++c) {
        if (!present[c]) continue;
        launch(ctx, k_ls_cflag, cdiv(m, kBlock), kBlock, 0, m, c, (const int32_t *)cls.p,
               (const int32_t *)g.eu.p, (const int32_t *)g.ev.p, (const int32_t *)label.p, flag.p);
        int64_t na = 0;
        scan_i64(ctx, flag.p, pos.p, m, &na);
        launch(ctx, k_ls_cfill, cdiv(m, kBlock), kBlock, 0, m, (const int64_t *)flag.p,
               (const int64_t *)pos.p, (const int32_t *)g.eu.p, (const int32_t *)g.ev.p,
               (const int32_t *)label.p, act[cur].p, ca[cur].p, cb[cur].p);
        for (int level = 0; na > 0; ++level) {
            if (++stamp == INT32_MAX) fail(GRASS_ERR_INVALID, "low-stretch tree: too many levels");
            memset_d(ctx, small.p + 2, 0, 2 * sizeof(int));
            launch(ctx, k_ls_xmark, cdiv(na, kBlock), kBlock, 0, na, (const int32_t *)ca[cur].p,
                   (const int32_t *)cb[cur].p, stamp, mark.p, xl.p, (unsigned int *)(small.p + 3),
                   small.p + 2, (unsigned long long)seed, c, level);
            d2h(ctx, hs, small.p, sizeof(hs));
            const int S = hs[2];
            const int64_t nx = (int64_t)(unsigned int)hs[3];
            launch(ctx, k_ls_xinit, cdiv(nx, kBlock), kBlock, 0, nx, (const int32_t *)xl.p,
                   (const int *)(small.p + 2), (unsigned long long)seed, c, level, ctr.p, when.p,
                   start.p, key.p, wb.p, eb.p);
            if (na <= ctx->lsst_small_level) {
                launch(ctx, k_ls_level, 1, kLevelBlock, 0, na, nx, (const int32_t *)act[cur].p,
                       (const int32_t *)ca[cur].p, (const int32_t *)cb[cur].p,
                       (const int32_t *)xl.p, (const int *)(small.p + 2), (const int32_t *)start.p,
                       (const double *)g.ew64.p, ctr.p, when.p, key.p, wb.p, eb.p, in_tree);
                edge_passes += 3 * (S + 1);
            }
            if (na > ctx->lsst_small_level && ctx->num_sms > 0) {
                int64_t na_ = na, nx_ = nx;
                const int32_t *act_ = act[cur].p, *ca_ = ca[cur].p, *cb_ = cb[cur].p, *xl_ = xl.p;
                const int *smax_ = small.p + 2;
                const int32_t *start_ = start.p;
                const double *ew_ = g.ew64.p;
                int32_t *ctr_ = ctr.p, *when_ = when.p, *eb_ = eb.p;
                unsigned long long *key_ = key.p, *wb_ = wb.p;
                uint8_t *tree_ = in_tree;
                unsigned int *bar = ctx->gbar.p;
                long long budget = ctx->wait_budget;
                int *err = ctx->flags.p + 3;
                const int grid = coop_grid(ctx, k_ls_level_grid, kLevelBlock, 0, na);
                GCK(cudaMemsetAsync(bar, 0, sizeof(unsigned int), ctx->stream));
                void *args[] = {&na_, &nx_, &act_, &ca_, &cb_, &xl_, &smax_, &start_, &ew_, &ctr_,
                                &when_, &key_, &wb_, &eb_, &tree_, &bar, &budget, &err};
                GCK(cudaLaunchCooperativeKernel((const void *)k_ls_level_grid, dim3(grid),
                                                dim3(kLevelBlock), args, 0, ctx->stream));
                ctx->launches++;
                edge_passes += 3 * (S + 1);
            }
            for (int t = 0; t <= S && na > ctx->lsst_small_level && ctx->num_sms == 0; ++t) {
                launch(ctx, k_ls_offer, cdiv(na, kBlock), kBlock, 0, na, (const int32_t *)ca[cur].p,
                       (const int32_t *)cb[cur].p, (const int32_t *)ctr.p, (const int32_t *)when.p,
                       (const int32_t *)start.p, t, key.p);
                launch(ctx, k_ls_heavy, cdiv(na, kBlock), kBlock, 0, na,
                       (const int32_t *)act[cur].p, (const int32_t *)ca[cur].p,
                       (const int32_t *)cb[cur].p, (const int32_t *)ctr.p, (const int32_t *)when.p,
                       (const int32_t *)start.p, t, (const unsigned long long *)key.p,
                       (const double *)g.ew64.p, wb.p);
                launch(ctx, k_ls_eid, cdiv(na, kBlock), kBlock, 0, na, (const int32_t *)act[cur].p,
                       (const int32_t *)ca[cur].p, (const int32_t *)cb[cur].p,
                       (const int32_t *)ctr.p, (const int32_t *)when.p, (const int32_t *)start.p, t,
                       (const unsigned long long *)key.p, (const double *)g.ew64.p,
                       (const unsigned long long *)wb.p, eb.p);
                launch(ctx, k_ls_commit, cdiv(nx, kBlock), kBlock, 0, nx, (const int32_t *)xl.p, t,
                       (const unsigned long long *)key.p, (const int32_t *)eb.p,
                       (const int32_t *)start.p, ctr.p, when.p, in_tree);
                edge_passes += 3;
            }
            rounds += S + 1;
            ++levels;
            launch(ctx, k_ls_relabel, cdiv(n, kBlock), kBlock, 0, n, (const int32_t *)ctr.p, label.p);
            launch(ctx, k_ls_nflag, cdiv(na, kBlock), kBlock, 0, na, (const int32_t *)ca[cur].p,
                   (const int32_t *)cb[cur].p, (const int32_t *)ctr.p, flag.p);
            int64_t nn = 0;
            scan_i64(ctx, flag.p, pos.p, na, &nn);
            launch(ctx, k_ls_nfill, cdiv(na, kBlock), kBlock, 0, na, (const int64_t *)flag.p,
                   (const int64_t *)pos.p, (const int32_t *)act[cur].p, (const int32_t *)ca[cur].p,
                   (const int32_t *)cb[cur].p, (const int32_t *)ctr.p, act[cur ^ 1].p,
                   ca[cur ^ 1].p, cb[cur ^ 1].p);
            cur ^= 1;
            na = nn;
        }
    }
    check_timeout(ctx);   // a level whose grid barrier gave up
    DBuf<unsigned long long> cnt;
    cnt.alloc(1);
    memset_d(ctx, cnt.p, 0, sizeof(unsigned long long));
    launch(ctx, k_ls_count, std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, cdiv(m, kBlock))),
           kBlock, 0, m, (const uint8_t *)in_tree, cnt.p);
    unsigned long long ne = 0;
    d2h(ctx, &ne, cnt.p, sizeof(ne));
    if ((int64_t)ne != n - 1)
        fail(GRASS_ERR_DISCONNECTED, "the graph is not connected (low-stretch forest has " +
                                         std::to_string(ne) + " edges for n - 1 = " +
                                         std::to_string(n - 1) + ")");
    if (stats) {
        stats->classes = nclass;
        stats->levels = levels;
        stats->rounds = rounds;
        stats->edge_passes = edge_passes;
    }
}

void tree_stretch(grass_ctx_t ctx, grass_tree_t T, double *st, double *total) {
    const GraphData &g = T->g;
    const int64_t n = g.n, m = g.m;
    if (!T->euler.built)
        fail(GRASS_ERR_INVALID, "stretch needs the tree's Euler tour (trees of at most euler_max_n vertices)");
    DBuf<int32_t> par, dep[2], anc;
    DBuf<double> res[2];
    DBuf<int> changed;
    par.alloc(n);
    dep[0].alloc(n);
    dep[1].alloc(n);
    res[0].alloc(n);
    res[1].alloc(n);
    changed.alloc(1);
    launch(ctx, k_st_rootinit, cdiv(n, kBlock), kBlock, 0, n, (const uint8_t *)T->isroot.p, par.p,
           res[0].p, dep[0].p);
    launch(ctx, k_st_parent, cdiv(m, kBlock), kBlock, 0, m, (const uint8_t *)T->in_tree.p,
           (const int32_t *)g.eu.p, (const int32_t *)g.ev.p, (const double *)g.ew64.p,
           (const int32_t *)T->euler.ein.p, par.p, res[0].p);
    // ancestor table anc[k*n + v] = the 2^k-th ancestor (a root stays put);
    // depth < 2^31, so 32 levels suffice
    constexpr int kMaxLevels = 32;
    anc.alloc((size_t)kMaxLevels * n);
    GCK(cudaMemcpyAsync(anc.p, par.p, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->stream));
    int cur = 0, K = 1;
    for (int k = 0; k + 1 < kMaxLevels; ++k) {
        memset_d(ctx, changed.p, 0, sizeof(int));
        launch(ctx, k_st_jump, cdiv(n, kBlock), kBlock, 0, n, (const int32_t *)(anc.p + (size_t)k * n),
               (const double *)res[cur].p, (const int32_t *)dep[cur].p, anc.p + (size_t)(k + 1) * n,
               res[cur ^ 1].p, dep[cur ^ 1].p, changed.p);
        cur ^= 1;
        int ch = 0;
        d2h(ctx, &ch, changed.p, sizeof(int));
        // no change: level k already maps every vertex to its root, and
        // res / dep hold the full sums to the root
        K = k + 1;
        if (!ch) break;
    }
    DBuf<double> stl;
    double *sp = st;
    if (!sp) {
        stl.alloc(m);
        sp = stl.p;
    }
    launch(ctx, k_st_edge, cdiv(m, kBlock), kBlock, 0, m, K, n, (const int32_t *)anc.p,
           (const int32_t *)g.eu.p, (const int32_t *)g.ev.p, (const double *)g.ew64.p,
           (const double *)res[cur].p, (const int32_t *)dep[cur].p, sp);
    if (total) {
        DBuf<double> part;
        part.alloc(kRedBlocks + 1);
        const int nb = (int)std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, cdiv(m, kBlock)));
        launch(ctx, k_st_part, nb, kBlock, 0, m, (const double *)sp, part.p);
        launch(ctx, k_st_final, 1, 32, 0, nb, (const double *)part.p, part.p + kRedBlocks);
        d2h(ctx, total, part.p + kRedBlocks, sizeof(double));
    }
    ctx->sync();
}

}  // namespace grass
