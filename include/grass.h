/*
 * grass.h -- C ABI of the GB300 sparsify-and-solve library.
 *
 * The library implements the data-parallel path of GRASS, similarity-aware
 * spectral graph sparsification (Z. Feng, arXiv 1911.04382), on one GPU:
 *
 *   grass_build_tree   maximum-weight spanning tree of L_G and its
 *                      elimination schedule                     (Sec. III-B, III-H)
 *   grass_embed        t-step generalized power iteration over r vectors
 *                      and the Joule heat of every off-sparsifier edge
 *                                                              (Sec. III-F, IV-B)
 *   grass_filter       threshold theta_sigma, optional top-K   (Eq. heatratio_final)
 *   grass_densify      iterative densification rounds          (Sec. IV-D)
 *   grass_pcg_solve    PCG on L_G + D preconditioned by L_S + D (Sec. V-A)
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - "device" pointers are CUDA device (or managed) memory on the device that
 *   was current when the context was created; "host" pointers are ordinary
 *   host memory.  The library never frees caller memory.
 * - Handles (context, tree, sparsifier) are opaque, owned by the library and
 *   released by the matching *_destroy call.  A tree or sparsifier is only
 *   valid with the context (and device) that created it.
 * - Every call enqueues its GPU work on the context's stream.  Calls that
 *   return host-side results (counts, scalars, statistics) synchronise that
 *   stream before returning; the others return as soon as work is enqueued.
 * - Every call returns a grass_status and never aborts, traps or exits.
 *   grass_last_error(ctx) gives a one-line description of the last failure.
 * - Vectors and blocks are row-major: block X of n rows and r columns holds
 *   X[i*r + j].  "prec" selects float (GRASS_FP32) or double (GRASS_FP64)
 *   element type for the void* blocks of a call.
 * - Edge ids: edge e = (u < v, w = -A(u,v)) is numbered by the rank of its
 *   upper-triangle entry in row-major order of the CSR (explicit zeros are
 *   not edges).
 */
#ifndef GRASS_H
#define GRASS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GRASS_OK = 0,
    GRASS_ERR_INVALID = 1,        /* bad argument or malformed / non-symmetric CSR  */
    GRASS_ERR_NOT_SDD = 2,        /* a row has D(p) = row sum < -1e-12 A(p,p)        */
    GRASS_ERR_DISCONNECTED = 3,   /* the graph has more than one component           */
    GRASS_ERR_OOM = 4,            /* device allocation failed                        */
    GRASS_ERR_NOT_CONVERGED = 5,  /* iteration limit reached; outputs still written  */
    GRASS_ERR_TIMEOUT = 6,        /* a bounded device-side wait expired               */
    GRASS_ERR_CUDA = 7            /* any other CUDA runtime error                     */
} grass_status;

typedef enum { GRASS_FP64 = 0, GRASS_FP32 = 1 } grass_prec;

#define GRASS_MAX_ROUNDS 16

/* Full symmetric CSR of the SDD matrix A = L_G + D (Sec. II-A, Eq.
 * formula_laplacian): rows sorted by column, no duplicates, off-diagonal
 * entries <= 0 (-w for an edge), diagonal present.  All pointers device. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t *rowptr;   /* [n+1], rowptr[0] = 0, rowptr[n] = nnz */
    const int32_t *col;      /* [nnz] */
    const double *val;       /* [nnz] */
} grass_csr_t;

/* Densification parameters (Sec. IV-D). */
typedef struct {
    double sigma2;               /* target relative condition number sigma^2          */
    int r;                       /* random vectors per round: 1, 2, 4, 8, 16, 24, 32  */
    int t;                       /* power steps per round, >= 1 (paper: t = 2)        */
    int max_rounds;              /* densification rounds, 1..GRASS_MAX_ROUNDS         */
    int lmax_iters;              /* power steps for the lambda_max estimate (< 10)    */
    int64_t max_add_per_round;   /* <= 0: keep every edge over the threshold          */
    grass_prec embed_prec;       /* precision of power iteration, SpMM and heat       */
    double inner_tol;            /* inner CG: stop at ||r|| <= inner_tol ||y||         */
    int inner_maxit;             /* inner CG: iteration cap                           */
} grass_params_t;

typedef struct {
    int rounds;                              /* filter+add passes executed            */
    int stopped_similar;                     /* 1 if lmax/lmin <= sigma^2 ended it    */
    int64_t added;                           /* off-tree edges added in total          */
    int64_t offtree_embedded;                /* off-S edges embedded, summed over rounds */
    int64_t added_round[GRASS_MAX_ROUNDS];
    int64_t embedded_round[GRASS_MAX_ROUNDS];
    double lmin_est[GRASS_MAX_ROUNDS];
    double lmax_est[GRASS_MAX_ROUNDS];
    double theta[GRASS_MAX_ROUNDS];
    double heat_max[GRASS_MAX_ROUNDS];
    int64_t inner_iters;                     /* inner CG iterations, all solves       */
    double ms_estimate, ms_embed, ms_filter, ms_update, ms_total;
    double ms_embed_round[GRASS_MAX_ROUNDS]; /* each round's power steps + heat (ms)  */
    int64_t lmax_capped[GRASS_MAX_ROUNDS];   /* inner solves of round k's lambda_max
                                                estimate that reached inner_maxit (0 or
                                                1: the estimate ends at the first)     */
} grass_sparsify_stats_t;

typedef struct {
    int iters;              /* PCG iterations (all refinement passes)          */
    int refinements;        /* FP64 refinement passes (FP32 mode), else 0       */
    int64_t inner_iters;    /* inner CG iterations of the preconditioner        */
    double rel_resid_fp64;  /* ||b - A x||_2 / ||b||_2 recomputed in FP64       */
    double ms;
} grass_solve_stats_t;

typedef struct grass_ctx_s *grass_ctx_t;
typedef struct grass_tree_s *grass_tree_t;
typedef struct grass_sparsifier_s *grass_sparsifier_t;

/* ---------------------------------------------------------------- context */

/* Create a context on the current CUDA device.  stream: a cudaStream_t
 * passed as void* (NULL = the legacy default stream).  The caller keeps
 * ownership of the stream.  Errors: INVALID (out == NULL), CUDA, OOM. */
grass_status grass_ctx_create(grass_ctx_t *out, void *stream);
void grass_ctx_destroy(grass_ctx_t ctx);
/* Switch the stream later calls enqueue on (same device). */
grass_status grass_ctx_set_stream(grass_ctx_t ctx, void *stream);
/* Text of the last failure of a call on ctx ("" if none).  Valid until the
 * next call on ctx. */
const char *grass_last_error(grass_ctx_t ctx);
/* Number of GPU kernel launches the library issued on ctx so far. */
int64_t grass_launch_count(grass_ctx_t ctx);

/* Bounded device-side waits (no counterpart in the paper).  The tree solve
 * runs as one cooperative kernel whose rounds are separated by grid
 * barriers; every barrier wait polls at most `polls` times (0 = default,
 * about one second) and then ends the kernel, and the call that launched it
 * returns GRASS_ERR_TIMEOUT with the context still usable.
 * hold_barriers != 0 is for testing that path: every barrier then waits for
 * one block more than the grid has, so every wait runs out.  Synchronises. */
grass_status grass_ctx_set_wait_limit(grass_ctx_t ctx, int64_t polls, int hold_barriers);

/* Launch-shape knobs (no counterpart in the paper), read by the kernels at
 * launch time.  Tree-solve results do not depend on them; the fused inner
 * CG groups its sums by block, so its results can change in the last bits
 * with the grid these knobs give.  Names:
 *   "tree_blocks_per_sm"  blocks per SM of the cooperative tree solve (1-8)
 *   "tree_threads"        threads per block of that kernel (128-1024, x32);
 *                         the fused PCG and the fused CG of the elimination
 *                         form with one column use at most 512 of them
 *   "tree_tail_items"     rounds at the end whose total work is below this
 *                         many items run in one block (work: surviving
 *                         vertices x max(1, r/4); default 2048; 0 = none)
 *   "euler_solve"         1 (default): grounded solves of L_T alone (no D)
 *                         with one column use the scan form (two segmented
 *                         prefix sums: along the Euler tour for a solve on
 *                         its own, over the preorder's vertex slots inside
 *                         the inner CG and the power steps, whose vectors
 *                         are then kept in preorder); 0: the elimination
 *                         rounds
 *   "similarity_check"    0 (default) or 1: grass_densify filters each
 *                         round's edges with the similarity check of
 *                         grass_filter_similar (Sec. IV-D step 6)
 *   "pcg_precond"         0 (default): grass_pcg_solve's preconditioner is the
 *                         tree solve / inner CG of inner_maxit; 1: one V-cycle
 *                         of the sparsifier's aggregation multigrid for
 *                         L_S + D (the sparsifier's solver; Sec. IV-C-1 and
 *                         IV-D step 1 name multigrid for it), a fixed SPD
 *                         preconditioner (plain PCG update), hierarchy built
 *                         on first use after each change of S; also used by
 *                         grass_fiedler's solves
 *   "amg_sweeps"          weighted-Jacobi sweeps before and after each
 *                         coarse correction of the V-cycle (1-8, default 1)
 *   "amg_fused"           1 (default): with one sweep, each multigrid PCG
 *                         pass runs as one cooperative kernel (every level,
 *                         the coarsest solve and the PCG scalars on the
 *                         device); 0: one launch per level step, replayed
 *                         as a CUDA graph
 *   "amg_warp_n"          levels of at most this many vertices (default
 *                         16384) take one warp per row in the fused kernel
 *   "amg_warp_setup_n"    the hierarchy's setup takes one warp per vertex
 *                         for its long-row steps on levels of at most this
 *                         many vertices (default 16384; the same hierarchy
 *                         as one thread per vertex)
 *   "amg_tail_n"          levels of at most this many vertices (default 0:
 *                         none but the coarsest dense solve) run in one
 *                         block of the fused kernel
 *   "lmax_amg"            0 (default) or 1: the lambda_max estimate's solves
 *                         with L_S (one column) are CG preconditioned by the
 *                         multigrid V-cycle of L_S, in FP64, to inner_tol
 *   "euler_max_n"         trees built on this context with more vertices
 *                         than this (default 4,000,000) get no Euler tour
 *                         and keep the elimination rounds (the tour's FP64
 *                         arrays then no longer fit the L2 cache and its
 *                         gathers are slower than the rounds)
 *   "spmm_variant"        -1 (default: the autotuner's choice, else 0) or
 *                         0-7: the r-column SpMM's launch variant, see
 *                         grass_autotune_rows
 *   "spmm_chunk"          -1 (default: the autotuner's choice, else the
 *                         widest), 0 (widest chunk the row and alignment
 *                         allow) or 16 (at most 16-byte chunks)
 *   "heat_lanes"          heat kernel form: 0 (default: several lanes per
 *                         edge when the row splits into 2 or 4 chunks), 1
 *                         (one lane per edge), 2 / 3 (forms 0 / 1 with two
 *                         edges in flight per lane); set by
 *                         grass_autotune_rows
 *   "lsst_small_level"    grass_build_lsst runs a level with at most this
 *                         many active edges in one block (default 4096;
 *                         measured at 100^3: 37.9 ms against 51.5 ms with
 *                         none and 49.2 ms at 32768); the tree is the same
 *   "grid_sms"            cooperative kernels (tree solves, fused CG and
 *                         PCG) use at most this many SMs (0, the default:
 *                         all); results depend on the grid, so a fixed
 *                         value gives fixed results
 * Errors: INVALID for an unknown name or a value out of range. */
grass_status grass_ctx_set_param(grass_ctx_t ctx, const char *name, int64_t value);

/* Kernel timing for roofline measurements (no counterpart in the paper).
 * family != GRASS_KF_NONE brackets every launch of that kernel family with
 * CUDA events on the context stream and accumulates, per launch, the
 * algorithmic bytes the launch must move (each array counted once per
 * phase that touches it):
 *   GRASS_KF_SPMM_G  Y = L_G X:  4(n+1) + 2m(4+s) + 2nrs
 *   GRASS_KF_SPMM_BLK  the launches of GRASS_KF_SPMM_G with r > 1 columns
 *                    (the embedding's power steps), same bytes
 *   GRASS_KF_SPMM_S  the same over the sparsifier's adjacency (+ns with D)
 *   GRASS_KF_HEAT    m_off(8+s) + nrs + m_off s
 *   GRASS_KF_TREE    one whole tree solve:
 *                    4nrs + receivers(16+2s) + (n-1)(16+4s)
 *   GRASS_KF_CG      one fused inner CG solve on the sparsifier: its
 *                    iterations (read back from the device) times
 *                    [tree solve + SpMV over S + 12nrs] plus 2nrs (+nrs
 *                    for max |X|, +2nrs for a preorder scatter)
 *   GRASS_KF_PCG     one fused PCG run (grass_pcg_solve, one launch per
 *                    refinement pass): its outer iterations times
 *                    [tree solve + SpMV with A + 12ns] (tree preconditioner),
 *                    [tree solve + SpMV with A + S's CSR + 14ns] (one inner
 *                    step, in closed form) or [SpMV with A + 15ns] plus the
 *                    inner CG iterations times [tree solve + SpMV over S +
 *                    12ns] (inner CG); plus 4ns (6ns with the inner CG)
 * (n rows, r columns, s = 4 or 8 bytes, m edges.)  Enabling resets the
 * accumulators.  grass_kernel_timing_read synchronises the stream and
 * returns the summed event time (ms), the number of timed launches and the
 * summed algorithmic bytes.  Timing adds two event records per launch. */
typedef enum {
    GRASS_KF_NONE = 0,
    GRASS_KF_SPMM_G = 1,
    GRASS_KF_SPMM_S = 2,
    GRASS_KF_HEAT = 3,
    GRASS_KF_TREE = 4,
    GRASS_KF_CG = 5,
    GRASS_KF_PCG = 6,
    GRASS_KF_SPMM_BLK = 7
} grass_kernel_family;
grass_status grass_kernel_timing_enable(grass_ctx_t ctx, int family);
grass_status grass_kernel_timing_read(grass_ctx_t ctx, double *ms, int64_t *launches, double *bytes);

/* ---------------------------------------------------------------- tree */

/* Validate A = L_G + D (Sec. II-A), extract its edges, build the
 * maximum-weight spanning tree (ties broken by smaller edge id, so the tree
 * is unique) and the tree's elimination schedule.  The paper's backbone is a
 * low-stretch tree (Sec. III-B); this library uses the maximum-weight tree.
 * ground: the row rho at which L_T and L_S are made invertible (the limit of
 * the tiny diagonal on one row, Sec. III-F); 0 <= ground < n.
 * The tree copies what it needs from A; A may be freed afterwards.
 * Errors: INVALID (bad CSR, positive or unmatched off-diagonal, n < 2,
 * nnz >= 2^31), NOT_SDD, DISCONNECTED, OOM, CUDA. */
grass_status grass_build_tree(grass_ctx_t ctx, const grass_csr_t *A, int32_t ground,
                              grass_tree_t *out);
void grass_tree_destroy(grass_tree_t tree);

/* The same as grass_build_tree with the caller's spanning tree in place of
 * the maximum-weight one: tree_eids (device, n-1 edge ids in any order) are
 * the tree's edges, e.g. the "hair-comb" tree of a 2D mesh (Sec. V-C) or a
 * low-stretch tree (Sec. III-B).  The ids are checked to lie in [0, m), to
 * be distinct and to form a spanning tree (no cycle); the graph must be
 * connected.  Everything after the tree (schedule, factors, sparsifiers,
 * solves) is as for grass_build_tree.  Errors: INVALID (bad CSR, ids out of
 * range, repeated, or containing a cycle), NOT_SDD, DISCONNECTED, OOM, CUDA. */
grass_status grass_tree_from_edges(grass_ctx_t ctx, const grass_csr_t *A, const int64_t *tree_eids,
                                   int32_t ground, grass_tree_t *out);

/* Low-stretch spanning tree in place of the maximum-weight one (Sec. III-B:
 * the backbone the paper starts from is a tree of low total stretch
 * st_T(G) = sum_e w_e R_T(e) = Tr(L_T^+ L_G)).  The construction clusters
 * by weight classes, heaviest first (class = the binade of w_e), and within
 * the edges of classes <= c repeats shifted low-diameter decompositions of
 * the cluster graph until every component is one cluster:
 *   shift(x) = 3 min(20, leading zeros of SplitMix64(seed + (x+1) G +
 *   (1000003 c + level) H)), G = 0x9E3779B97F4A7C15, H = 0xD1B54A32D192ED03;
 *   a cluster starts growing at round S - shift(x) (S the largest shift);
 *   an unclaimed cluster next to clusters claimed in the previous round
 *   joins the centre with the smallest (start, centre id) through the
 *   heaviest edge (smallest id on equal weight) to such a neighbour; that
 *   edge joins the tree; clusters are then renamed by their centres.
 * The result is a function of (graph, seed) alone: runs and devices agree
 * bit for bit.  Everything after the tree is as for grass_build_tree.
 * stats (host, may be NULL): classes, decompositions ("levels") and growth
 * rounds run, and the construction's device time in ms (CUDA events).
 * Errors: as grass_build_tree. */
typedef struct {
    int32_t classes;
    int64_t levels;
    int64_t rounds;
    double ms;
} grass_lsst_stats_t;
grass_status grass_build_lsst(grass_ctx_t ctx, const grass_csr_t *A, uint64_t seed, int32_t ground,
                              grass_tree_t *out, grass_lsst_stats_t *stats);

/* Stretch of every edge of the tree's graph, w_e times the resistance of
 * the tree path between its endpoints (tree edges: 1), into stretch
 * (device, m doubles, may be NULL), and their sum st_T(G) (host, may be
 * NULL; a deterministic FP64 sum).  Single trees only, of at most
 * euler_max_n vertices (the tree's Euler tour orients it).  Errors: INVALID
 * (a forest, or no Euler tour), OOM, CUDA. */
grass_status grass_tree_stretch(grass_ctx_t ctx, grass_tree_t tree, double *stretch, double *total);

/* Sizes: n, m (edges), factor_rounds (contraction rounds of the tree
 * elimination schedule).  Any pointer may be NULL.  Host outputs. */
grass_status grass_tree_info(grass_tree_t tree, int64_t *n, int64_t *m, int64_t *factor_rounds);

/* Per-round sizes of the elimination schedule (host outputs, room for cap
 * rounds each, any may be NULL): vertices eliminated, vertices receiving
 * updates, and updates (contributions), round by round. */
grass_status grass_tree_schedule_info(grass_tree_t tree, int64_t *eliminated, int64_t *receivers,
                                      int64_t *contributions, int64_t cap);

/* Export the extracted graph (device outputs, m entries each, any may be
 * NULL): eu[e] < ev[e], ew[e] = w_e; D (n entries) = diagonal load. */
grass_status grass_tree_graph(grass_ctx_t ctx, grass_tree_t tree, int32_t *eu, int32_t *ev,
                              double *ew, double *D);

/* Export in_tree[e] = 1 for tree edges, else 0 (device, m bytes). */
grass_status grass_tree_edges(grass_ctx_t ctx, grass_tree_t tree, uint8_t *in_tree);

/* X = L_T^{-1} B grounded at rho (with_D = 0; X[rho] = 0) or
 * X = (L_T + D)^{-1} B (with_D = 1), by the tree's elimination schedule
 * (Sec. III-H: linear-time tree factorization).  B, X: device, n x r.
 * B and X may alias.  r in {1, 2, 4, 8, 16, 24, 32} (other values: INVALID). */
grass_status grass_tree_solve(grass_ctx_t ctx, grass_tree_t tree, int with_D, int r,
                              grass_prec prec, const void *B, void *X);

/* The same solve as grass_tree_solve, same arguments and results, with no
 * device-memory allocation.  The paper has no counterpart: this entry exists
 * for callers that cannot let a library allocate once they run (a fixed
 * device-memory budget already handed to another allocator, or a loop that
 * must not call cudaMalloc/cudaFree because they synchronise the device).
 *   Scratch: a 256-byte array compiled into the library (grid-barrier
 * counter and wait-timeout flag), held by every GPU that loads the library
 * until the process exits.  Its size does not grow with the tree; the one
 * limit it sets is that the cooperative grid times the schedule's grid
 * barriers stays below 2^31 (far above any schedule the library builds);
 * beyond it the call returns GRASS_ERR_INVALID.
 *   Set-up: the first call in a CUDA context (once per device, and again
 * after the application resets the device) looks up the array's address
 * there (cudaGetSymbolAddress); make that first call before any stream
 * capture.  This note concerns the set-up only.
 *   Sharing: every call on a device uses the same array, which keeps the
 * last call's contents; each call zeroes it on ctx's stream before its
 * kernel and copies in ctx's barrier-hold setting (grass_ctx_set_wait_limit).  Calls that overlap on the GPU (other streams, contexts or
 * threads on the same device) race on it: order them.
 *   with_D = 1 needs the L_T + D factor, which is built (allocated) by a
 * first grass_tree_solve with with_D = 1; without it the call returns
 * GRASS_ERR_INVALID.  The call waits for its kernel (it reads the timeout
 * flag back): GRASS_ERR_TIMEOUT as for grass_tree_solve.  Other errors:
 * INVALID for bad arguments, CUDA for a failed launch. */
grass_status grass_tree_solve_noalloc(grass_ctx_t ctx, grass_tree_t tree, int with_D, int r,
                                      grass_prec prec, const void *B, void *X);

/* Y = L_G X (graph Laplacian, D excluded; Eq. formula_laplacian).
 * X, Y: device, n x r, must not alias.  r in {1, 2, 4, 8, 16, 24, 32}. */
grass_status grass_spmm(grass_ctx_t ctx, grass_tree_t tree, int r, grass_prec prec,
                        const void *X, void *Y);

/* ---------------------------------------------------------------- sparsifier */

/* New sparsifier S = the tree (Sec. III-B step 1). */
grass_status grass_sparsifier_create(grass_ctx_t ctx, grass_tree_t tree, grass_sparsifier_t *out);
void grass_sparsifier_destroy(grass_sparsifier_t S);
/* Add edges (device ids, count >= 0) to S.  Ids already in S are ignored;
 * ids out of range give INVALID. */
grass_status grass_sparsifier_add(grass_ctx_t ctx, grass_sparsifier_t S, const int64_t *eids,
                                  int64_t count);
/* Host outputs: edges in S, edges outside S (m_off). */
grass_status grass_sparsifier_info(grass_sparsifier_t S, int64_t *n_edges, int64_t *m_off);
/* in_s[e] = 1 if edge e is in S (device, m bytes). */
grass_status grass_sparsifier_mask(grass_ctx_t ctx, grass_sparsifier_t S, uint8_t *in_s);
/* Host export of the sparsifier's edge set (Sec. IV-D: the sparsifier that
 * densification returns, the preconditioner of Sec. V-A): the ids of the
 * edges in S in increasing order.  eids_host: host, room for cap ids (may be
 * NULL when cap = 0); the first min(cap, count) ids are written.  *count
 * (host) = the number of edges in S.  Uses S's context and stream;
 * synchronises.  Errors: INVALID (null S or count, cap < 0), CUDA. */
grass_status grass_sparsifier_edges(grass_sparsifier_t S, int64_t *eids_host, int64_t cap,
                                    int64_t *count);
/* Ids of the edges outside S, increasing (device, m_off entries): the order
 * of the heat array of grass_embed. */
grass_status grass_sparsifier_offtree(grass_ctx_t ctx, grass_sparsifier_t S, int64_t *eids);

/* ---------------------------------------------------------------- embed / filter */

/* Spectral embedding of the off-S edges (Sec. III-F, Eqs. formula_pwr_iter,
 * formula_pwr_iter5new, formula_pwr_iter6):
 *   H <- L_S^{-1} L_G H, t times, from H = h0 (n x r, device, double);
 * L_S^{-1} grounded at rho; by the tree solve when S is the tree, else by
 * r-column CG on L_S preconditioned by the tree (inner_tol, inner_maxit).
 * After each step H is multiplied by the power of two that puts max|H| in
 * [1,2) (exact; the common factor leaves normalised heats unchanged).
 * h0 need not be orthogonal to 1: the first product with L_G removes any
 * constant.  Outputs (device, optional = NULL):
 *   H_out [n x r] in prec;  heat [m_off] in prec, heat[i] = w_e sum_j
 *   (H[u][j] - H[v][j])^2 for the i-th off-S edge e = (u,v) in increasing id.
 * Host output heat_max (optional).  r in {1, 2, 4, 8, 16, 24, 32}, t >= 1. */
grass_status grass_embed(grass_ctx_t ctx, grass_sparsifier_t S, const double *h0, int r, int t,
                         grass_prec prec, double inner_tol, int inner_maxit, void *H_out,
                         void *heat, double *heat_max);

/* lambda_min estimate (Sec. IV-C-2, Eq. formula_courant-fischer-3):
 * min over p of L_G(p,p) / L_S(p,p), Laplacian diagonals.  Host output. */
grass_status grass_lambda_min(grass_ctx_t ctx, grass_sparsifier_t S, double *lmin);

/* lambda_max estimate (Sec. IV-C-1): iters generalized power steps from v0
 * (device, n doubles), then the Rayleigh quotient v^T L_G v / v^T L_S v
 * (FP64 sums).  Host output. */
grass_status grass_lambda_max(grass_ctx_t ctx, grass_sparsifier_t S, const double *v0, int iters,
                              grass_prec prec, double inner_tol, int inner_maxit, double *lmax);

/* Edge filter (Eq. formula_heatratio_final):
 *   theta = (sigma2 * lmin / lmax)^(2t+1); keep off-S edge i iff
 *   heat[i] >= theta * max(heat).
 * cap > 0 keeps at most cap edges, the largest heats first and the smaller
 * id among equal heats (radix select).  heat: device [m_off] in prec, the
 * order of grass_embed.  accepted: device, room for min(m_off, cap) ids,
 * written in increasing id.  Host outputs n_accepted, theta (optional). */
grass_status grass_filter(grass_ctx_t ctx, grass_sparsifier_t S, const void *heat, grass_prec prec,
                          double sigma2, double lmin, double lmax, int t, int64_t cap,
                          int64_t *accepted, int64_t *n_accepted, double *theta);

/* Edge filter with the similarity check of Sec. IV-D step 6 ("only add
 * dissimilar edges"), which the paper leaves undefined; read here as an
 * endpoint conflict: of the off-S edges grass_filter would keep without a
 * cap (heat >= theta * max(heat)), take them in order of heat descending,
 * smaller id first among equal heats, and reject every edge with an
 * endpoint on an edge kept before it; then cap > 0 keeps the first cap of
 * the kept ones in that order.  The kept edges form a matching.  Arguments,
 * outputs and errors as grass_filter.  grass_densify applies the same check
 * after grass_ctx_set_param(ctx, "similarity_check", 1). */
grass_status grass_filter_similar(grass_ctx_t ctx, grass_sparsifier_t S, const void *heat,
                                  grass_prec prec, double sigma2, double lmin, double lmax, int t,
                                  int64_t cap, int64_t *accepted, int64_t *n_accepted,
                                  double *theta);

/* ---------------------------------------------------------------- densify / solve */

/* Iterative densification (Sec. IV-D).  Per round k < max_rounds:
 * (2) lambda estimates on the current S, (3) stop if lmax/lmin <= sigma2
 * and every inner CG solve of the lambda_max estimate met inner_tol before
 * inner_maxit (a Rayleigh quotient after inexact solves can fall far below
 * lambda_max; the estimate's power steps end at the first solve that did
 * not, and stats->lmax_capped[k] is then 1),
 * (4) embed with h0 + k*n*r (device, max_rounds*n*r doubles) and the
 * lambda_max start v0 + k*n (device, max_rounds*n doubles), (5) filter by
 * theta_sigma, add the kept edges.  theta_sigma takes the round's
 * lambda_max estimate when its solves converged, else the last estimate
 * whose solves did (round 1's are direct tree solves): lambda_max can only
 * fall as edges are added.  stats->lmax_est[k] is the round's own estimate,
 * stats->theta[k] the theta_sigma used.  The paper's step (6) similarity check is applied when
 * the context's "similarity_check" parameter is 1 (grass_filter_similar).
 * out: a new sparsifier (tree + added edges).  stats: host, optional. */
grass_status grass_densify(grass_ctx_t ctx, grass_tree_t tree, const grass_params_t *params,
                           const double *h0, const double *v0, grass_sparsifier_t *out,
                           grass_sparsify_stats_t *stats);

/* Solve A x = b, A = L_G + D of the tree's matrix, by PCG (Sec. V-A),
 * x0 = 0, until ||b - A x||_2 <= tol ||b||_2 (measured in FP64).
 * Preconditioner M = L_S + D: the tree solve when S is the tree (or when
 * inner_maxit = 0), else r=1 CG on L_S + D preconditioned by the tree
 * (inner_tol, inner_maxit) and the flexible PCG update.  Each PCG run is
 * one cooperative kernel (no host round trip per iteration).  prec = GRASS_FP64: FP64 PCG.  prec = GRASS_FP32:
 * FP32 vectors and matrix, FP64 dot products and alpha/beta, wrapped in FP64
 * iterative refinement (each pass reduces the residual by refine_tol).
 * b, x: device, n doubles.  maxit bounds PCG iterations over all passes.
 * Errors: NOT_CONVERGED (x and stats still written).  stats optional. */
grass_status grass_pcg_solve(grass_ctx_t ctx, grass_sparsifier_t S, const double *b, double *x,
                             double tol, int maxit, grass_prec prec, double refine_tol,
                             double inner_tol, int inner_maxit, grass_solve_stats_t *stats);

/* ---------------------------------------------------------------- partitioning */

typedef struct {
    int iters_done;          /* inverse power iterations run                    */
    int64_t pcg_iters;       /* PCG iterations over all of them                 */
    double worst_rel_resid;  /* largest FP64 relative residual of a solve       */
    int64_t n_pos, n_neg;    /* vertices on each side of the sign cut           */
    double rayleigh;         /* u^T L_G u of the returned unit vector u         */
    double ms;
} grass_fiedler_stats_t;

/* Spectral graph partitioning (Sec. V-F, Table VI): an approximate Fiedler
 * vector by `iters` inverse power iterations on A = L_G + D of S's tree
 * (u <- A^{-1} u, each solve by grass_pcg_solve's PCG preconditioned by the
 * sparsifier, to ||b - A y|| <= tol ||b|| within maxit iterations, prec and
 * inner_maxit as there), with u made orthogonal to the all-ones vector and
 * normalised to unit length before and after every solve (for a graph
 * Laplacian, D = 0, this keeps the singular system consistent), then the
 * sign cut side[i] = 1 iff u[i] >= 0.
 *   x0: device, n doubles (the start vector; need not be orthogonal to 1).
 *   u_out: device, n doubles (the final unit vector), optional.
 *   side_out: device, n bytes, optional.  stats: host, optional.
 * Errors: INVALID, NOT_CONVERGED (some solve missed tol; outputs and stats
 * still written), TIMEOUT, CUDA. */
grass_status grass_fiedler(grass_ctx_t ctx, grass_sparsifier_t S, const double *x0, int iters,
                           double tol, int maxit, grass_prec prec, int inner_maxit, double *u_out,
                           uint8_t *side_out, grass_fiedler_stats_t *stats);

/* ---------------------------------------------------------------- batching */

/* Batched form (no counterpart in the paper, which handles one graph at a
 * time): many independent graphs stored as one block-diagonal matrix A (the
 * union CSR, graph k on rows [seg_off[k], seg_off[k+1]), no entry joining
 * two graphs).  grass_build_forest extracts every graph, builds the maximum
 * spanning tree of each (a spanning forest, Sec. III-B) with the graph's
 * first vertex as its root, and one elimination schedule over the whole
 * forest (Sec. III-H): every later launch serves all graphs at once.
 * seg_off: host, nseg+1 entries, seg_off[0] = 0, seg_off[nseg] = n, every
 * graph >= 2 vertices.  Errors as grass_build_tree; DISCONNECTED when some
 * graph is; INVALID when an edge joins two graphs.
 * On a forest, grass_tree_solve solves every graph (each grounded at its
 * root), grass_spmm and grass_embed work edge by edge (grass_embed's
 * heat_max is then the maximum over all graphs), and the per-graph calls
 * are the *_batch ones below; grass_lambda_min/max, grass_filter,
 * grass_densify and grass_pcg_solve return INVALID. */
grass_status grass_build_forest(grass_ctx_t ctx, const grass_csr_t *A, int64_t nseg,
                                const int64_t *seg_off, grass_tree_t *out);
/* Number of graphs and their vertex and edge-id ranges (host outputs of
 * nseg+1 entries, any may be NULL).  A tree from grass_build_tree is one
 * graph. */
grass_status grass_tree_segments(grass_tree_t tree, int64_t *nseg, int64_t *vtx_off,
                                 int64_t *edge_off);
/* One densification round (Sec. IV-D steps 1-5) for every graph of a
 * forest at once: per graph lambda_min (Eq. courant-fischer-3), lambda_max
 * (lmax_iters power steps from v0, Rayleigh quotient), the stop test
 * lambda_max / lambda_min <= sigma^2, theta_sigma (Eq. heatratio_final);
 * one embedding of r vectors over the whole batch (h0, v0: as
 * grass_densify, n rows of the union); each graph keeps its off-tree edges
 * with heat >= theta_k * heat_max_k.  P->max_rounds must be 1 and
 * P->max_add_per_round <= 0.  stats: aggregate (min lambda_min, max
 * lambda_max, smallest theta, largest heat_max).  per_graph: host, optional,
 * 6 doubles per graph: lambda_min, lambda_max, theta (inf: similar, nothing
 * added), heat_max, edges added, off-tree edges embedded.  Reductions of a
 * graph run over ranges of its own rows and edges in a fixed order, so its
 * results do not depend on the other graphs of the batch. */
grass_status grass_densify_batch(grass_ctx_t ctx, grass_tree_t forest, const grass_params_t *P,
                                 const double *h0, const double *v0, grass_sparsifier_t *out,
                                 grass_sparsify_stats_t *stats, double *per_graph);
/* PCG (Sec. V-A) on every graph of the batch at once, x0 = 0, each graph
 * with its own scalars, until ||b_k - A_k x_k||_2 <= tol ||b_k||_2 measured
 * in FP64 for every graph.  Preconditioner M = L_S + D of the graph: the
 * forest solve, then inner_maxit CG steps on L_S + D preconditioned by it
 * (flexible outer update).  prec: vectors in FP64 or FP32; dot products and
 * scalars FP64.  FP64 iterative refinement: after a pass, the graphs whose
 * FP64 residual r = b - A x still misses tol run another pass on A e = r
 * (x += e in FP64); stats->refinements counts the passes (at most 8).
 * One outer iteration is captured into a CUDA graph and replayed when the
 * context's stream can be captured (not the legacy default stream, kernel
 * timing off).  b, x: device, n doubles.  stats: iters = most iterations of
 * any graph, rel_resid_fp64 = largest.  iters_per_graph (int32) and
 * rel_resid (double): host, nseg entries, optional.  NOT_CONVERGED when
 * some graph misses tol within maxit iterations (outputs still written). */
grass_status grass_pcg_solve_batch(grass_ctx_t ctx, grass_sparsifier_t S, const double *b,
                                   double *x, double tol, int maxit, grass_prec prec,
                                   int inner_maxit, grass_solve_stats_t *stats,
                                   int32_t *iters_per_graph, double *rel_resid);
/* Autotuner (no counterpart in the paper): time the tree (forest) solve of
 * r columns under each launch shape -- threads per block {256, 512, 1024},
 * blocks per SM {1, 2, 4}, shared-memory tail {1024, 4096, 16384} items --
 * and keep the fastest on ctx (as grass_ctx_set_param would).  best: host
 * [3] = threads, blocks per SM, tail items; best_ms: host, its time per
 * solve.  Results of every solve are the same under any shape. */
grass_status grass_autotune(grass_ctx_t ctx, grass_tree_t tree, int r, grass_prec prec,
                            int64_t *best, double *best_ms);
/* Row-kernel autotuner (no counterpart in the paper): on the tree's graph,
 * time the r-column SpMM (Y = L_G X) under each launch variant -- neighbour
 * batch {by row size, 1, 2, 4} x register cap {none, 6 blocks per SM}, and
 * each block on a contiguous range of rows (batch by row size or 1) -- and
 * each chunk width {widest, 16 bytes}, and the Joule-heat kernel of the
 * tree's off-tree edges in each of its forms ("heat_lanes"); keep the
 * fastest on ctx: the SpMM choice for (prec, r) (the "spmm_variant" and
 * "spmm_chunk" knobs, when set, still take precedence), the heat form as
 * the "heat_lanes" knob.  best: host [3] = chunk cap (0 = widest, 16),
 * variant (0-7), heat form (0-3); best_ms: host [2] = SpMM and heat time
 * per launch.  Results are the same up to rounding order under any choice.
 * Errors: INVALID, OOM, CUDA. */
grass_status grass_autotune_rows(grass_ctx_t ctx, grass_tree_t tree, int r, grass_prec prec,
                                 int32_t *best, double *best_ms);

/* ---------------------------------------------------------------- serving */

/* Serving form (no counterpart in the paper, which solves one system at a
 * time on one core): a request loop that runs whole sparsify-and-solve
 * requests -- grass_build_tree (ground 0), grass_densify, grass_pcg_solve --
 * for many callers on one GPU.
 *   Admission: `slots` worker threads, each with its own context on its own
 * non-blocking stream.  Requests are taken in arrival order; the oldest
 * waiting request is admitted as soon as a slot is idle and its footprint
 * (grass_server_footprint) fits in what the device-memory budget has left,
 * and the ones behind it wait for it.  A request whose footprint exceeds
 * the whole budget is refused at submission (OOM).
 *   State: an admitted request keeps its inputs, tree, sparsifier and
 * Krylov vectors on the device until it completes, and frees them then.
 * Requests in flight run concurrently on their slots' streams.
 *   Results: launch shapes depend on each request alone, so a request's x
 * and statistics are the same whether it runs alone or among others.
 * Times are host seconds since the server was created. */
typedef struct grass_server_s *grass_server_t;

typedef struct {
    /* host inputs: the caller keeps them alive until grass_server_wait on
     * the ticket returns */
    int64_t n, nnz;
    const int64_t *rowptr;      /* [n+1] full symmetric CSR of L_G + D        */
    const int32_t *col;         /* [nnz]                                       */
    const double *val;          /* [nnz]                                       */
    const double *h0;           /* [max_rounds * n * r] grass_densify's h0     */
    const double *v0;           /* [max_rounds * n]     grass_densify's v0     */
    const double *b;            /* [n] right-hand side                         */
    double *x;                  /* [n] host output, written before completion  */
    grass_params_t params;      /* densification parameters                    */
    double tol;                 /* PCG: ||b - A x|| <= tol ||b||              */
    int maxit;
    grass_prec pcg_prec;
    double refine_tol, pcg_inner_tol;
    int pcg_inner_maxit;
} grass_request_t;

typedef struct {
    grass_status status;        /* of the first failing call, else GRASS_OK    */
    char error[128];            /* its grass_last_error text                   */
    grass_sparsify_stats_t sparsify;
    grass_solve_stats_t solve;
    int64_t footprint_bytes;    /* what admission reserved for it              */
    double t_submit, t_admit, t_done;   /* seconds since grass_server_create   */
    double ms_h2d, ms_tree, ms_densify, ms_pcg;   /* phases, host wall time    */
    int slot;                   /* worker that ran it                          */
    int in_flight_at_admit;     /* requests running once it was admitted        */
} grass_result_t;

/* Start `slots` (1..64) workers on CUDA device `device`.  hbm_budget: bytes
 * of device memory requests may reserve in total (<= 0: 85 % of the memory
 * free now; capped at the memory free now).  Errors: INVALID, CUDA, OOM. */
grass_status grass_server_create(int device, int slots, int64_t hbm_budget, grass_server_t *out);
/* The budget in bytes (-1 for a null server). */
int64_t grass_server_budget(grass_server_t srv);
/* Server-wide knob applied to every request admitted after the call:
 * "grid_sms" = the context knob of that name on each worker (0: all SMs;
 * a share such as SMs / slots lets admitted requests' cooperative kernels
 * run side by side).  Errors: INVALID (unknown name, value out of range). */
grass_status grass_server_set_param(grass_server_t srv, const char *name, int64_t value);
/* Queue a request (copied; its host arrays are read when it is admitted).
 * *ticket identifies it for grass_server_wait.  Errors: INVALID (bad
 * request, or the server is stopping), OOM (footprint above the budget). */
grass_status grass_server_submit(grass_server_t srv, const grass_request_t *req, int64_t *ticket);
/* Block until the request completes; *out gets its result and the ticket
 * is released.  Errors: INVALID (unknown ticket). */
grass_status grass_server_wait(grass_server_t srv, int64_t ticket, grass_result_t *out);
/* Host snapshot: reserved bytes, requests queued and running, and the most
 * requests that ran at once so far.  Any pointer may be NULL. */
grass_status grass_server_stats(grass_server_t srv, int64_t *in_use, int64_t *queued,
                                int64_t *running, int64_t *max_running);
/* Wait for every queued and running request, stop the workers, free all. */
void grass_server_destroy(grass_server_t srv);
/* Device bytes admission reserves for a request with n rows, nnz stored
 * entries, r vectors and `rounds` densification rounds: its inputs and an
 * upper bound of the library's allocations.  Host only (no GPU needed);
 * -1 for invalid sizes. */
int64_t grass_server_footprint(int64_t n, int64_t nnz, int r, int rounds);

#ifdef __cplusplus
}
#endif
#endif /* GRASS_H */
