// common.cuh -- internal definitions shared by the CUDA sources of the
// library: error handling, launch accounting, device buffers, the block
// layout used by every r-column kernel, and the handle structs.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/grass.h"

namespace grass {

// ---------------------------------------------------------------- errors

struct Error {
    grass_status st;
    std::string msg;
};

[[noreturn]] inline void fail(grass_status st, const std::string &msg) { throw Error{st, msg}; }

inline void check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return;
    cudaGetLastError();   // clear a sticky launch error if any
    fail(e == cudaErrorMemoryAllocation ? GRASS_ERR_OOM : GRASS_ERR_CUDA,
         std::string(what) + ": " + cudaGetErrorString(e));
}

#define GCK(call) ::grass::check_cuda((call), #call)

// ---------------------------------------------------------------- buffers

// Owning device buffer (synchronous cudaMalloc/cudaFree; long-lived data).
template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count) {
        release();
        if (count == 0) count = 1;
        GCK(cudaMalloc((void **)&p, count * sizeof(T)));
        n = count;
    }
    // grow-only
    void reserve(size_t count) {
        if (count <= n && p) return;
        alloc(count);
    }
    T *get() const { return p; }
};

// A device array carved from an Arena (not owning).
template <typename T>
struct ASpan {
    T *p = nullptr;
    size_t n = 0;
};

// Bump allocation from device chunks of at least 64 MB, freed together: one
// cudaMalloc per chunk instead of one per array (and no synchronising
// cudaFree per array).  reset() reuses the chunks from the start.
struct Arena {
    std::vector<std::unique_ptr<DBuf<char>>> chunks;
    size_t cur = 0, off = 0;
    void reset() { cur = off = 0; }
    size_t bytes() const {
        size_t b = 0;
        for (const auto &c : chunks) b += c->n;
        return b;
    }
    template <typename T>
    T *get(size_t count) {
        const size_t bytes = ((count ? count : 1) * sizeof(T) + 255) & ~(size_t)255;
        while (cur < chunks.size() && off + bytes > chunks[cur]->n) {
            ++cur;
            off = 0;
        }
        if (cur == chunks.size()) {
            auto c = std::make_unique<DBuf<char>>();
            c->alloc(bytes > ((size_t)64 << 20) ? bytes : ((size_t)64 << 20));
            chunks.push_back(std::move(c));
            off = 0;
        }
        T *q = reinterpret_cast<T *>(chunks[cur]->p + off);
        off += bytes;
        return q;
    }
    template <typename T>
    void get(ASpan<T> &a, size_t count) {
        a.p = get<T>(count);
        a.n = count ? count : 1;
    }
};

// ---------------------------------------------------------------- context

enum ScratchSlot {
    SCR_SCAN = 0, SCR_SCAN2, SCR_TMP0, SCR_TMP1, SCR_TMP2, SCR_TMP3,
    SCR_Y, SCR_H, SCR_CG_X, SCR_CG_R, SCR_CG_Z, SCR_CG_P, SCR_CG_Q,
    SCR_PCG_X, SCR_PCG_R, SCR_PCG_Z, SCR_PCG_P, SCR_PCG_Q, SCR_PCG_ZOLD, SCR_PCG_E,
    SCR_FILTER, SCR_FILTER2, SCR_HEAT, SCR_LMAX_V, SCR_LMAX_Y, SCR_PART2,
    SCR_EU_S, SCR_EU_C, SCR_EU_P, SCR_EU_A, SCR_CG_XP,
    SCR_SIM_V, SCR_SIM_E, SCR_SIM_C,
    SCR_PART_X, SCR_PART_Y, SCR_PART_1, SCR_AMG_Y, SCR_AMG_X, SCR_ONES,
    SCR_COUNT
};

// device scalar area layout (doubles)
enum {
    DS_ITER = 40,        // inside DS_RED: inner-CG iteration accumulator
    DS_CAPPED = 41,      // inside DS_RED: inner-CG solves that reached their iteration cap
    DS_PCG = 42,         // inside DS_RED: fused PCG iterations and final r.r
    DS_RED = 0,          // 64 doubles: reduction outputs (PCG scalars)
    DS_CG = 64,          // 12 x 32 doubles: per-column CG scalars
    DS_MAX = 448,        // 16 x uint64: max-abs bit patterns
    DS_TOTAL = 512
};

}  // namespace grass

struct grass_ctx_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int64_t launches = 0;
    grass::DBuf<int> flags;                 // device error flags
    grass::DBuf<double> scal;               // device scalars (DS_*)
    grass::DBuf<double> partials;           // block partial sums
    grass::DBuf<unsigned int> counters;     // last-block counters
    double *hpin = nullptr;                 // pinned host staging (4096 doubles)
    grass::DBuf<char> scratch[grass::SCR_COUNT];
    // bounded device waits: barrier state and poll budget (flags[3] = timeout)
    grass::DBuf<unsigned int> gbar;
    long long wait_budget = 1LL << 23;   // polls; about 0.15 us each on GB300
    int num_sms = 0;
    // launch-shape knobs (grass_ctx_set_param)
    int tree_bpsm = 1;
    int grid_sms = 0;      // cooperative grids on at most this many SMs (0: all)
    int heat_lanes = 0;    // heat kernel form (0-3), see blk.cu heat_T
    int64_t lsst_small_level = 4096;   // low-stretch levels run in one block up to this many edges
    // SpMM launch variant (0..7) and chunk cap (0 = widest, 16) when >= 0;
    // else spmm_tuned[fp64][r slot] = {chunk cap, variant} from the autotuner
    int spmm_variant = -1, spmm_chunk = -1;
    int spmm_tuned[2][7][2] = {};
    int tree_threads = 1024;
    int64_t tree_tail_items = 2048;
    int euler_solve = 1;   // scan form for grounded r = 1 solves without D
    int similarity_check = 0;   // 1: Sec. IV-D step 6 in grass_densify (endpoint conflicts)
    int pcg_precond = 0;        // 1: the sparsifier's multigrid V-cycle preconditions PCG
    int amg_sweeps = 1;         // Jacobi sweeps before and after each coarse correction
    int lmax_amg = 0;           // 1: lambda_max estimates solve L_S by multigrid-preconditioned CG
    grass::Arena amg_tmp;       // the multigrid setup's temporary arrays
    int amg_fused = 1;          // 1: the multigrid PCG runs as one cooperative kernel (amg_fused.cu)
    int64_t amg_tail_n = 0;     // its levels of at most this many vertices run in one block
    int64_t amg_warp_n = 16384; // its levels of at most this many vertices take a warp per row
    int64_t amg_warp_setup_n = 16384;   // hierarchy setup: levels of at most this many
                                        // vertices use the warp forms of the long-row kernels
    // a non-blocking stream of the context's own, on which multi-kernel
    // iterations are captured into CUDA graphs and replayed (ordered with the
    // caller's stream by events); created on first use
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t cap_ev[2] = {nullptr, nullptr};
    int64_t euler_max_n = 4000000;   // trees larger than this keep the elimination rounds
    // co-resident grid of each cooperative kernel shape, per context (no
    // process-wide state: contexts may run on different host threads)
    struct CoopEntry {
        const void *kernel;
        int threads;
        size_t smem;
        int bpsm;
        int grid;   // co-resident blocks per SM
    };
    std::vector<CoopEntry> coop_cache;
    // kernel-family timing (grass_kernel_timing_*)
    int tfam = 0;
    std::vector<cudaEvent_t> events;
    size_t ev_used = 0;
    int64_t t_launches = 0;
    double t_bytes = 0.0;

    // launches whose bytes scale with a device-side iteration count: bytes =
    // fixed + per_iter * (counter after - counter before)
    struct IterLaunch {
        double fixed, per_iter;
        size_t slot;
    };
    std::vector<IterLaunch> iter_launches;
    grass::DBuf<double> iter_snap;      // [2 * launches] counter before / after

    bool t_begin(int fam, double bytes) {
        if (fam == 0 || fam != tfam) return false;
        while (events.size() < ev_used + 2) {
            cudaEvent_t e;
            GCK(cudaEventCreate(&e));
            events.push_back(e);
        }
        GCK(cudaEventRecord(events[ev_used], stream));
        t_bytes += bytes;
        t_launches += 1;
        return true;
    }
    // snapshot of a device double counter into slot 2k (+1 for "after")
    void t_snap(const double *counter, size_t k, int after) {
        if (iter_snap.n < 2 * (k + 1)) {
            grass::DBuf<double> nb;
            nb.alloc(std::max<size_t>(64, 4 * (k + 1)));
            if (iter_snap.p)
                GCK(cudaMemcpyAsync(nb.p, iter_snap.p, iter_snap.n * sizeof(double),
                                    cudaMemcpyDeviceToDevice, stream));
            GCK(cudaStreamSynchronize(stream));
            std::swap(nb.p, iter_snap.p);
            std::swap(nb.n, iter_snap.n);
        }
        GCK(cudaMemcpyAsync(iter_snap.p + 2 * k + after, counter, sizeof(double),
                            cudaMemcpyDeviceToDevice, stream));
    }
    void t_end(bool timed) {
        if (!timed) return;
        GCK(cudaEventRecord(events[ev_used + 1], stream));
        ev_used += 2;
    }
    ~grass_ctx_s() {
        for (auto e : events) cudaEventDestroy(e);
        for (auto e : cap_ev)
            if (e) cudaEventDestroy(e);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }

    template <typename T>
    T *scr(int slot, size_t count) {
        size_t bytes = count * sizeof(T);
        auto &b = scratch[slot];
        if (b.n < bytes || !b.p) {
            GCK(cudaStreamSynchronize(stream));
            b.alloc(bytes + 256);
        }
        return reinterpret_cast<T *>(b.p);
    }
    void sync() { GCK(cudaStreamSynchronize(stream)); }
};

namespace grass {

// ---------------------------------------------------------------- launches

template <typename... KArgs, typename... Args>
inline void launch(grass_ctx_t ctx, void (*kernel)(KArgs...), int64_t grid, int block, size_t smem,
                   Args &&...args) {
    if (grid <= 0) return;
    if (grid > 2147483647LL) fail(GRASS_ERR_INVALID, "grid too large");
    kernel<<<(unsigned)grid, block, smem, ctx->stream>>>(std::forward<Args>(args)...);
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) check_cuda(e, "kernel launch");
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

constexpr int kBlock = 256;
constexpr int kRedBlocks = 608;     // 4 x 152 SMs: fixed grid for deterministic reductions
// Contraction rounds are O(log n) in practice (23 for a million-vertex
// spanning tree); solves keep the per-round offsets in shared memory.
constexpr int kMaxRounds = 512;
// shared memory for the tail of a tree solve (vertices x columns x element)
constexpr size_t kTailSmem = 184 * 1024;   // + up to ~40 KB static shared memory <= 227 KB
constexpr int kPersistMaxThreads = 1024;
// The fused Krylov kernels whose preconditioner is the elimination-round
// solve (the PCG, the inner CG with D or r > 1 columns of the non-scan form)
// hold more live values than 64 registers a thread: at most 512 threads per
// block, so that a thread may keep 128 registers instead of spilling.
constexpr int kFusedMaxThreads = 512;
constexpr int64_t kAmgCoarse = 256;   // the multigrid's coarsest level has at most this many vertices
constexpr int kAmgFusedLevels = 24;   // levels the fused multigrid PCG takes (kernel parameters)
// threads of a persistent kernel launched with the knob value but bounded
// by the kernel's own maximum
inline int bounded_threads(int knob, int bound) { return knob < bound ? knob : bound; }

// ---------------------------------------------------------------- block layout
// An n x R row-major block is processed by TPR consecutive threads per row,
// each owning EPT consecutive elements: consecutive threads touch consecutive
// memory, and TPR divides 32 so a row never straddles a warp.
template <int R>
struct Lay {
    static constexpr int TPR = (R % 8 == 0) ? 8 : (R % 4 == 0) ? 4 : (R % 2 == 0) ? 2 : 1;
    static constexpr int EPT = R / TPR;
};

// Dispatch a functor templated on R over the supported column counts.
#define GRASS_DISPATCH_R(r, FN, ...)                                         \
    switch (r) {                                                             \
        case 1: FN<1>(__VA_ARGS__); break;                                   \
        case 2: FN<2>(__VA_ARGS__); break;                                   \
        case 4: FN<4>(__VA_ARGS__); break;                                   \
        case 8: FN<8>(__VA_ARGS__); break;                                   \
        case 16: FN<16>(__VA_ARGS__); break;                                 \
        case 24: FN<24>(__VA_ARGS__); break;                                 \
        case 32: FN<32>(__VA_ARGS__); break;                                 \
        default: ::grass::fail(GRASS_ERR_INVALID, "r must be 1, 2, 4, 8, 16, 24 or 32"); \
    }

inline bool r_supported(int r) {
    return r == 1 || r == 2 || r == 4 || r == 8 || r == 16 || r == 24 || r == 32;
}

// ---------------------------------------------------------------- graph / tree data

// Rows of an adjacency with more than kHeavyDeg entries (the hubs of a
// power-law graph): the r-column products give each one a whole block
// instead of the few lanes of an ordinary row (list order is arbitrary; every
// row's result is order-independent).
constexpr int kHeavyDeg = 256;
struct HeavyRows {
    int64_t count = 0;
    DBuf<int32_t> rows;
    DBuf<unsigned int> cnt;
};

struct GraphData {
    int64_t n = 0, m = 0;
    DBuf<int32_t> adj_ptr;            // [n+1] off-diagonal adjacency in CSR order
    DBuf<int32_t> adj_col;            // [2m]
    DBuf<int32_t> adj_eid;            // [2m]
    DBuf<double> adj_w64;             // [2m] w > 0
    DBuf<float> adj_w32;
    DBuf<int32_t> eu, ev;             // [m] edges, eu < ev
    DBuf<double> ew64;                // [m]
    DBuf<float> ew32;
    DBuf<double> D64;                 // [n] diagonal load
    DBuf<float> D32;
    DBuf<double> degG;                // [n] weighted degree (Laplacian diagonal)
    HeavyRows heavy;                  // rows of adj_ptr above kHeavyDeg entries
    bool lap_only = false;            // D = 0 everywhere: A is a graph Laplacian (singular)
    // a batch of independent graphs stored as one block-diagonal matrix:
    // graph k owns vertices [seg_voff[k], seg_voff[k+1]) and edge ids
    // [seg_eoff[k], seg_eoff[k+1]); one segment for a single graph
    int64_t nseg = 1;
    std::vector<int64_t> seg_voff, seg_eoff;   // host [nseg+1]
    DBuf<int32_t> seg_of;             // [n] graph of each vertex (nseg > 1 only)
    DBuf<int64_t> seg_voff_d;         // device copy of seg_voff (nseg > 1 only)
};

struct alignas(32) Dbl4 {
    double x, y, z, w;
};

// Elimination schedule of the spanning tree by rake (degree 1) and compress
// (degree 2) rounds; numeric factors for L_T (lap) and L_T + D (sdd).
struct TreeFactor {
    DBuf<double> invd64, b1_64, b2_64, cm64, fill64;
    DBuf<float> invd32, b1_32, b2_32, cm32;
    DBuf<double> rinv64;              // [nroots] 1 / pivot of each root (0: grounded)
    DBuf<float> rinv32;
    // packed per-item coefficients matching fwd_rec / bwd_rec
    DBuf<double2> fm64;               // [n_rcv] multipliers of the first two contributions
    DBuf<float2> fm32;
    DBuf<Dbl4> bc64;                  // [n - nroots] {1/d, w1/d, w2/d, 0} by elimination position
    DBuf<float4> bc32;
};

struct TreeSchedule {
    int rounds = 0;
    std::vector<int64_t> elim_off;   // host [rounds+1] into elim_list
    std::vector<int64_t> rcv_off;    // host [rounds+1] into rcv_list
    DBuf<int32_t> elim_list;         // [n - nroots]
    DBuf<int32_t> n1, n2;            // [n] neighbours at elimination (-1: none)
    DBuf<int32_t> src1, src2;        // [n] weight source: >= 0 tree edge id, < 0: fill of vertex -src-1
    DBuf<int32_t> rcv_list;          // receivers grouped by round
    DBuf<int32_t> rcv_beg;           // [#rcv + 1] start into contrib arrays
    DBuf<int32_t> contrib_v;         // contributor vertex
    DBuf<uint8_t> contrib_side;      // 0: receiver is n1 of v, 1: n2
    int64_t n_rcv = 0, n_contrib = 0;
    DBuf<int64_t> d_offs;            // device copy: rcv_off then elim_off
    // packed records, one load per item:
    DBuf<int4> fwd_rec;              // [n_rcv] {u, v0, v1 (-1), index of 3rd contribution (-1)}
    DBuf<int4> bwd_rec;              // [n - nroots] by elimination position {v, n1, n2 (-1), 0}
    // shared-memory tail: the vertices alive at round tail_k0 get local ids
    // 0..tail_n-1 in elimination order (the roots last, in root order);
    // records with local ids.
    int tail_k0 = 0;
    int64_t tail_n = 0;
    int64_t tail_c0 = 0;             // first contribution index of round tail_k0
    std::vector<int64_t> contrib_off;   // host [rounds+1]: first contribution of each round
    DBuf<int32_t> tail_vid;          // [tail_n] global id of each local id
    DBuf<int4> fwd_loc;              // [n_rcv - rcv_off[tail_k0]]
    DBuf<int4> bwd_loc;              // [n - nroots - elim_off[tail_k0]]
    DBuf<int32_t> contrib_loc;       // local id of contributors from round tail_k0 on
};

// Euler tour of the spanning tree (forest) for the scan form of the
// grounded solve (D = 0): tour[p] = v at the entry into v, -(v+1) at the
// exit; ein/eout the two positions of v (-1 for a root); pw the weight of
// v's edge to its parent.
struct EulerTour {
    bool built = false;
    int64_t L = 0;                   // 2 (n - nroots) positions
    DBuf<int32_t> tour, ein, eout;
    DBuf<uint8_t> head;              // [L] 1 at each tree's first position
    DBuf<double> pw;
    DBuf<double> ipw;                // [n] 1 / pw (roots: 1)
    DBuf<float> ipw32;
    // Preorder numbering (every tree: its root, then its vertices in the
    // order the tour enters them; trees in vertex-offset order): pre[v],
    // vert[k] = v, and the tour and per-vertex arrays in that numbering, for
    // solvers that keep their vectors in preorder (the tour's entry values
    // are then read in sequence).
    DBuf<int32_t> pre, vert, tour_pre, ein_pre, eout_pre;
    DBuf<uint8_t> head_pre;          // [n] 1 at every tree's root slot
    DBuf<double> ipw_pre;
    DBuf<float> ipw32_pre;
};

// Aggregation multigrid hierarchy of the sparsifier's matrix L_S (+ D)
// (amg.cu).  Level 0 is S itself; each coarser level is the exact Galerkin
// product P^T M P for the piecewise-constant aggregation P: the contracted
// graph (edges between different aggregates kept, repeated pairs kept as
// separate entries) with the aggregates' summed diagonal loads.
struct AmgLevel {
    int64_t n = 0, nnz = 0;
    ASpan<int32_t> ptr, col;          // off-diagonal adjacency (a column may repeat)
    ASpan<double> w64, diag64, D64;   // weights, diagonal = weighted degree + D, D
    ASpan<float> w32, diag32;
    ASpan<int32_t> agg;               // [n] coarse vertex of each vertex (not on the coarsest)
    ASpan<int32_t> aggcol;            // [nnz] agg[col[j]] (not on the coarsest)
    ASpan<int32_t> mptr, mem;         // members of coarse vertex c: mem[mptr[c] .. mptr[c+1])
    ASpan<char> vb, vx, vt;           // V-cycle vectors of this level (coarse levels)
};

struct AmgHier {
    Arena arena;                      // every level's arrays
    std::vector<std::unique_ptr<AmgLevel>> lv;
    bool singular = false;            // D = 0: the coarsest solve is grounded
    int64_t nc = 0;                   // coarsest size
    DBuf<double> cinv64;              // coarsest (grounded) inverse, dense row-major
    DBuf<float> cinv32;
    DBuf<char> t0;                    // level-0 scratch vector
};

// PCG on A = L_G + D with one V-cycle of H per iteration, one cooperative
// launch (amg_fused.cu); returns the iterations
template <typename T>
int amg_pcg_fused(grass_ctx_t ctx, grass_sparsifier_t S, AmgHier &H, const T *rhs, T *e,
                  double tol_abs, int maxit);

}  // namespace grass

struct grass_tree_s {
    grass_ctx_t ctx = nullptr;
    int32_t ground = 0;                // roots_h[0]
    // one root (grounded row) per graph: a spanning tree, or a spanning
    // forest with one tree per graph of a batch
    int64_t nroots = 1;
    std::vector<int32_t> roots_h;
    grass::DBuf<int32_t> roots;        // [nroots]
    grass::DBuf<uint8_t> isroot;       // [n]
    grass::GraphData g;
    grass::DBuf<uint8_t> in_tree;     // [m]
    grass::TreeSchedule sched;
    grass::EulerTour euler;
    grass::TreeFactor lap;            // L_T grounded at rho
    grass::TreeFactor sdd;            // L_T + D
    bool has_sdd = false;
};

struct grass_sparsifier_s {
    grass_ctx_t ctx = nullptr;
    grass_tree_t tree = nullptr;
    bool is_tree = true;
    int64_t n_edges = 0, m_off = 0;
    grass::DBuf<uint8_t> in_s;        // [m]
    grass::DBuf<int32_t> off_u, off_v, off_eid;   // [m_off] increasing id
    grass::DBuf<double> off_w64;
    grass::DBuf<float> off_w32;
    grass::DBuf<int32_t> s_ptr, s_col;            // S adjacency (when !is_tree)
    int64_t s_nnz = 0;
    grass::HeavyRows s_heavy;                     // rows of s_ptr above kHeavyDeg entries
    grass::DBuf<double> s_w64;
    grass::DBuf<float> s_w32;
    grass::DBuf<double> degS;         // [n]
    // S's adjacency with vertices renumbered in the tree's preorder (rows in
    // preorder, each row's entries in their original order); built on first
    // use after each change of S
    bool pre_ok = false;
    grass::DBuf<int32_t> p_ptr, p_col;
    grass::DBuf<double> p_w64;
    grass::DBuf<float> p_w32;
    // multigrid hierarchies of L_S ([0]) and L_S + D ([1]), built on first
    // use after each change of S
    std::unique_ptr<grass::AmgHier> amg[2];
};

namespace grass {

// ---------------------------------------------------------------- util API (util.cu)

// out[0..n] = exclusive prefix sums of in[0..n-1]; out[n] = total.  Host
// receives the total when total_host != nullptr (synchronises).
void scan_i64(grass_ctx_t ctx, const int64_t *in, int64_t *out, int64_t n, int64_t *total_host);

struct U64x2 {
    unsigned long long a, b;
};
void scan_pair(grass_ctx_t ctx, const U64x2 *in, U64x2 *out, int64_t n, U64x2 *total_host);

// out[j] = sum_i A[i*r+j] * B[i*r+j] (double accumulation, deterministic),
// written to device doubles out[0..r).
void dot_cols(grass_ctx_t ctx, int r, grass_prec prec, int64_t n, const void *A, const void *B,
              double *out);
// Pulls `count` doubles from device to host (synchronises).
void d2h(grass_ctx_t ctx, void *dst, const void *src, size_t bytes);
void h2d(grass_ctx_t ctx, void *dst, const void *src, size_t bytes);
void memset_d(grass_ctx_t ctx, void *p, int v, size_t bytes);
// v -= mean(v) (FP64, deterministic sum): the projection on the complement
// of the all-ones vector, the range of a graph Laplacian
void project_ones(grass_ctx_t ctx, int64_t n, double *v);
void copy_d(grass_ctx_t ctx, void *dst, const void *src, size_t bytes);

// ---------------------------------------------------------------- per-module entry points

void graph_extract(grass_ctx_t ctx, const grass_csr_t *A, GraphData &g);
void mst_boruvka(grass_ctx_t ctx, const GraphData &g, uint8_t *in_tree);
void mst_boruvka_w(grass_ctx_t ctx, const GraphData &g, const double *ew, uint8_t *in_tree);
// Low-stretch spanning tree (lsst.cu): in_tree (device, m bytes) of the
// deterministic class-by-class shifted-decomposition construction; stats
// may be null.
struct LsstStats {
    int classes = 0;
    int64_t levels = 0, rounds = 0, edge_passes = 0;
};
void lsst_build(grass_ctx_t ctx, const GraphData &g, uint64_t seed, uint8_t *in_tree,
                LsstStats *stats);
// Per-edge stretch w_e R_T(u_e, v_e) (device, m doubles, may be null) and
// its sum (host, may be null); needs the tree's Euler tour.
void tree_stretch(grass_ctx_t ctx, grass_tree_t T, double *st, double *total);
void tree_schedule(grass_ctx_t ctx, grass_tree_t T);
// Euler tour from the tree adjacency (slot lists tptr/tocc, tree edge id of
// every slot in tsrc; L slots), before the contraction rounds modify it.
void euler_build(grass_ctx_t ctx, grass_tree_t T, const int32_t *tptr, const int32_t *tocc,
                 const int32_t *tsrc, int64_t L);
void tree_factor(grass_ctx_t ctx, grass_tree_t T, bool with_D, TreeFactor &f);
// In-place tree solve of the n x r block Y (prec); optionally tracks the
// max |x| bit pattern into maxbits (device, uint64 for both precisions).
void tree_solve_inplace(grass_ctx_t ctx, grass_tree_t T, const TreeFactor &f, int r,
                        grass_prec prec, void *Y, unsigned long long *maxbits);

// Y = scale * (L X + Dopt .* X) over an adjacency (ptr, col, w).  scale may
// come from a device max-bits word (pow2 rescale) when scale_from != nullptr.
void lap_mm(grass_ctx_t ctx, int r, grass_prec prec, int64_t n, int64_t nnz, const int32_t *ptr,
            const int32_t *col, const void *w, const void *Dopt, const void *X, void *Y,
            const unsigned long long *scale_from, int fam, const HeavyRows *hv);
// Row-kernel autotuner (blk.cu): SpMM launch variant and chunk width, heat
// kernel form, timed on the tree's graph; kept on ctx.  best: [3] chunk cap,
// variant, heat form; best_ms: [2] SpMM and heat ms per launch.
void autotune_rows(grass_ctx_t ctx, grass_tree_t T, int r, grass_prec prec, int32_t *best,
                   double *best_ms);
// hv.rows / hv.count for an adjacency (n rows, nnz entries); synchronises.
void heavy_rows(grass_ctx_t ctx, int64_t n, int64_t nnz, const int32_t *ptr, HeavyRows &hv);
// Convert an n x r double block to prec (copy or float conversion).
void convert_block(grass_ctx_t ctx, grass_prec prec, int64_t count, const double *src, void *dst);
// Multiply an n x r block in place by the pow2 factor derived from maxbits.
void apply_pow2(grass_ctx_t ctx, grass_prec prec, int64_t count, void *X,
                const unsigned long long *maxbits);
// heat over off-S edges; scale from maxbits; heat_max bits (uint64) written.
void heat_offs(grass_ctx_t ctx, int r, grass_prec prec, grass_sparsifier_t S, const void *H,
               const unsigned long long *scale_from, void *heat, unsigned long long *heatmax_bits);
// quadratic forms over all edges and over S edges for a single vector (r=1)
void quad_forms(grass_ctx_t ctx, grass_prec prec, grass_sparsifier_t S, const void *x,
                double *qG_qS_dev);
void max_abs_bits(grass_ctx_t ctx, grass_prec prec, int64_t count, const void *X,
                  unsigned long long *maxbits);

// ---------------------------------------------------------------- krylov.cu

// X = L_S^{-1} Y (grounded, or (L_S + D)^{-1} Y when with_D), r columns, by
// the tree solve (S is the tree) or tree-preconditioned CG.  Y is preserved
// unless S is the tree (then Y may be X).  Returns inner iterations (max over
// columns).  maxbits: optional max|X| tracking.
int64_t s_solve(grass_ctx_t ctx, grass_sparsifier_t S, bool with_D, int r, grass_prec prec,
                const void *Y, void *X, double tol, int maxit, unsigned long long *maxbits);

void pcg_solve(grass_ctx_t ctx, grass_sparsifier_t S, const double *b, double *x, double tol,
               int maxit, grass_prec prec, double refine_tol, double inner_tol, int inner_maxit,
               grass_solve_stats_t *st);

// ---------------------------------------------------------------- amg.cu

// The hierarchy of L_S (+ D with with_D), built on first use (S must not be
// the tree alone).
grass::AmgHier &amg_get(grass_ctx_t ctx, grass_sparsifier_t S, bool with_D);
// z = V-cycle(r): one multigrid V-cycle on L_S (+ D) from zero, r and z
// device vectors of n elements in prec (may not alias).
void amg_vcycle(grass_ctx_t ctx, grass_sparsifier_t S, bool with_D, grass_prec prec, const void *r,
                void *z);
// PCG on A = L_G + D with the V-cycle of L_S + D as the preconditioner, from
// e = 0, until ||rhs - A e|| <= tol_abs (maxit iterations at most); one
// iteration is captured into a CUDA graph and replayed.  Returns iterations.
template <typename T>
int amg_pcg(grass_ctx_t ctx, grass_sparsifier_t S, const T *rhs, T *e, double tol_abs, int maxit);
// x = L_S^+ y (D = 0; y projected on the complement of 1) by CG
// preconditioned by the V-cycle, until ||r|| <= tol ||y||; FP64; returns
// iterations (maxit when the cap was reached).
int amg_cg_lap(grass_ctx_t ctx, grass_sparsifier_t S, const double *y, double *x, double tol,
               int maxit);

// ---------------------------------------------------------------- api.cu helpers

double now_ms();
unsigned long long *maxslot(grass_ctx_t ctx, int k);
double bits_to_double(unsigned long long b);
void clear_timeout(grass_ctx_t ctx);
void check_timeout(grass_ctx_t ctx);
void ensure_sdd(grass_ctx_t ctx, grass_tree_t T);
int64_t power_steps(grass_ctx_t ctx, grass_sparsifier_t S, const double *h0, int r, int t,
                    grass_prec prec, double inner_tol, int inner_maxit, void *H, void *Y,
                    int *scale_slot);
double theta_sigma(double sigma2, double lmin, double lmax, int t);
grass_sparsifier_t new_sparsifier(grass_ctx_t ctx, grass_tree_t T);

// ---------------------------------------------------------------- sparsifier ops (filter.cu)

void sparsifier_rebuild(grass_ctx_t ctx, grass_sparsifier_t S);
void sparsifier_add(grass_ctx_t ctx, grass_sparsifier_t S, const int64_t *eids, int64_t count);
void lambda_min(grass_ctx_t ctx, grass_sparsifier_t S, double *out_host);
int64_t filter_heat(grass_ctx_t ctx, grass_sparsifier_t S, const void *heat, grass_prec prec,
                    double thr, int64_t cap, int64_t *accepted);
// Sec. IV-D step 6 (similarity check), endpoint-conflict reading: of the
// off-S edges with heat >= thr, keep those that the greedy pass in (heat
// descending, id ascending) order accepts when it rejects every edge with an
// endpoint on an edge accepted before it, then at most cap (> 0) of them, the
// first ones in that order.  Writes the kept ids (increasing) to accepted.
int64_t filter_similar(grass_ctx_t ctx, grass_sparsifier_t S, const void *heat, grass_prec prec,
                       double thr, int64_t cap, int64_t *accepted);

// A thread's dot-product accumulator.  Double vectors: an FP64 sum, as in
// the plain definition.  Float vectors: a pair of floats, the running sum and
// its accumulated error, adding the exact rounding error of every product
// (an FMA) and of every sum (two-sum): about 48 significant bits per thread
// with no FP64 arithmetic per element (on GB300 FP64 runs at a small
// fraction of the FP32 rate and was most of the time of the vector phases).
// Partials go on to the FP64 block and grid sums.
template <typename T>
struct Acc;
template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add_prod(double a, double b) { s += a * b; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float pe = __fmaf_rn(a, b, -p);   // a b = p + pe exactly
        const float t = __fadd_rn(hi, p);
        const float bp = __fsub_rn(t, hi);
        const float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));   // hi + p = t + se
        hi = t;
        lo = __fadd_rn(lo, __fadd_rn(se, pe));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ---------------------------------------------------------------- grid barrier
// Barrier for cooperative (co-resident) launches; bar[0] counts arrivals.
// Every wait is bounded: after `budget` polls, or
// as soon as another block has flagged an error, the block sets *err and
// leaves; the caller returns from the kernel, so a lost block can never hang
// the GPU.  All threads of a block get the same answer.
// bar[0] only grows within a launch (the host zeroes it before each launch):
// barrier number b is complete once bar[0] >= (b+1) * gridDim.x, so a block
// needs one release-add and then polls, with no reset round trip.
// bar[2] != 0 (testing only) raises every target by one arrival that never
// comes, so every wait runs out.
__device__ inline unsigned int ld_relaxed_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ inline void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ inline void red_add_release_u32(unsigned int *p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// `epoch` counts the barriers this block has passed in the launch (all
// blocks pass the same barriers, so barrier b completes when the counter
// reaches (b+1) * gridDim.x).  Arrival: one release reduction by thread 0,
// which carries the block's writes (ordered before it by __syncthreads).
// Wait: relaxed polls of the counter, back to back (the error flag and the
// poll budget are looked at every 64 polls), then one acquire fence, which pairs with
// the other blocks' release reductions.  The testing flag is read after
// the arrival, while the other blocks arrive.
__device__ inline bool grid_sync(unsigned int *bar, long long budget, int *err,
                                 unsigned int &epoch) {
    __shared__ int s_ok;
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
        int ok = 1;
        red_add_release_u32(bar, 1u);
        const unsigned int hold = ld_relaxed_u32(bar + 2) ? 1u : 0u;
        const unsigned int target = epoch * gridDim.x + hold;
        long long spins = 0;
        while (ld_relaxed_u32(bar) < target) {
            if ((++spins & 63) == 0) {
                if (*(volatile int *)err) {
                    ok = 0;
                    break;
                }
                if (spins > budget) {
                    atomicOr(err, 1);
                    ok = 0;
                    break;
                }
            }
        }
        fence_acq_rel_gpu();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// block-wide max of a non-negative double, one atomicMax on its bit pattern
__device__ inline void block_atomic_max(unsigned long long *maxbits, double v) {
    __shared__ double sm[32];
    for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, d));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? sm[lane] : 0.0;
        for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, d));
        if (lane == 0 && v > 0.0) atomicMax(maxbits, (unsigned long long)__double_as_longlong(v));
    }
}

// bits helpers
__host__ __device__ inline double pow2_scale_from_bits(unsigned long long maxbits_f64) {
    // maxbits holds the bit pattern of a non-negative double m; the factor
    // 2^-(floor(log2 m)) puts m in [1, 2).  m == 0 or non-finite: 1.
    unsigned long long ex = (maxbits_f64 >> 52) & 0x7FFULL;
    if (ex == 0 || ex == 0x7FF) return 1.0;
    long long e = (long long)ex - 1023;             // m = 1.f * 2^e
    unsigned long long bits = (unsigned long long)(1023 - e) << 52;   // 2^-e
    if (1023 - e <= 0 || 1023 - e >= 2047) return 1.0;
    double s;
    memcpy(&s, &bits, sizeof(s));
    return s;
}

}  // namespace grass
