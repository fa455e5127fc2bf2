// solve.cu -- stand-alone tree solves X = (L_T + D)^{-1} Y (or grounded),
// in place, by the elimination schedule of tree.cu.  One cooperative launch
// per solve (tree_solve.cuh); devices without cooperative launch get one
// launch per round instead.
#include "tree_solve.cuh"

namespace grass {

template <typename T, int R>
__global__ void __launch_bounds__(kPersistMaxThreads, 1)
    k_tree_persist(TreeKArgs<T> a, T *Y, unsigned long long *maxbits) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned int epoch = 0;
    double mx = 0.0;
    tree_tail_stage<T, R>(a, reinterpret_cast<T *>(smem_raw));
    if (!tree_solve_dev<T, R>(a, Y, epoch, mx, reinterpret_cast<T *>(smem_raw))) return;
    if (maxbits) block_atomic_max(maxbits, mx);
}

// scan form: grounded solve of L_T alone, one column
template <typename T>
__global__ void __launch_bounds__(kPersistMaxThreads, 1)
    k_euler_persist(EulerKArgs e, TreeKArgs<T> a, T *Y, unsigned long long *maxbits) {
    unsigned int epoch = 0;
    double mx = 0.0;
    if (!euler_solve_dev<T>(e, Y, a.bar, a.budget, a.err, epoch, mx)) return;
    if (maxbits) block_atomic_max(maxbits, mx);
}

// ---------------------------------------------------------------- per-round path

template <typename T, int R>
__global__ void k_fwd_round(int64_t r0, int64_t cnt, const int4 *rec, const typename PackT<T>::V2 *fm,
                            const int32_t *beg, const int32_t *cv, const T *cm, T *Y) {
    constexpr int TPR = Lay<R>::TPR;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = t / TPR;
    if (i >= cnt) return;
    fwd_packed<T, R>(r0 + i, (int)(t % TPR), rec[r0 + i], fm[r0 + i], beg, cv, cm, Y);
}

template <typename T, int R>
__global__ void k_bwd_round(int64_t e0, int64_t cnt, const int4 *rec,
                            const typename PackT<T>::V4 *bc, T *Y, unsigned long long *maxbits) {
    constexpr int TPR = Lay<R>::TPR;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = t / TPR;
    double mx = 0.0;
    if (i < cnt) mx = bwd_packed<T, R>((int)(t % TPR), rec[e0 + i], bc[e0 + i], Y);
    if (maxbits) block_atomic_max(maxbits, mx);
}

template <typename T, int R>
__global__ void k_root(const int32_t *roots, const T *root_invd, T *Y, unsigned long long *maxbits) {
    double mx = 0.0;
    const int64_t rho = roots[blockIdx.x];   // one block per root
    if (threadIdx.x < R) {
        T v = root_invd[blockIdx.x] * Y[rho * R + threadIdx.x];
        Y[rho * R + threadIdx.x] = v;
        mx = fabs((double)v);
    }
    if (maxbits) block_atomic_max(maxbits, mx);
}

template <typename T, int R>
static void solve_rounds(grass_ctx_t ctx, grass_tree_t Tr, const TreeKArgs<T> &a, T *Y,
                         unsigned long long *maxbits) {
    constexpr int TPR = Lay<R>::TPR;
    const TreeSchedule &S = Tr->sched;
    for (int k = 0; k < S.rounds; ++k) {
        int64_t r0 = S.rcv_off[k], cnt = S.rcv_off[k + 1] - r0;
        launch(ctx, k_fwd_round<T, R>, cdiv(cnt * TPR, kBlock), kBlock, 0, r0, cnt, a.fwd_rec, a.fm,
               a.beg, a.cv, a.cm, Y);
    }
    launch(ctx, k_root<T, R>, Tr->nroots, 32, 0, (const int32_t *)Tr->roots.p, a.root_invd, Y, maxbits);
    for (int k = S.rounds - 1; k >= 0; --k) {
        int64_t e0 = S.elim_off[k], cnt = S.elim_off[k + 1] - e0;
        launch(ctx, k_bwd_round<T, R>, cdiv(cnt * TPR, kBlock), kBlock, 0, e0, cnt, a.bwd_rec, a.bc,
               Y, maxbits);
    }
}

// ---------------------------------------------------------------- dispatch

template <typename T, int R>
static void solve_T(grass_ctx_t ctx, grass_tree_t Tr, const TreeFactor &f, T *Y,
                    unsigned long long *maxbits) {
    size_t smem = 0;
    TreeKArgs<T> a = tree_kargs<T, R>(ctx, Tr, f, &smem);
    if (ctx->num_sms <= 0) {
        solve_rounds<T, R>(ctx, Tr, a, Y, maxbits);
        return;
    }
    const int threads = ctx->tree_threads;
    if (R == 1 && &f == &Tr->lap && ctx->euler_solve && Tr->euler.built) {
        const int grid = coop_grid(ctx, k_euler_persist<T>, threads, 0, Tr->g.n);
        EulerKArgs e;
        euler_kargs<T>(ctx, Tr, grid, &e);
        GCK(cudaMemsetAsync(a.bar, 0, sizeof(unsigned int), ctx->stream));
        void *eargs[] = {&e, &a, &Y, &maxbits};
        GCK(cudaLaunchCooperativeKernel((const void *)k_euler_persist<T>, dim3(grid),
                                        dim3(threads), eargs, 0, ctx->stream));
        ctx->launches++;
        return;
    }
    const int grid = coop_grid(ctx, k_tree_persist<T, R>, threads, smem, Tr->g.n * Lay<R>::TPR);
    GCK(cudaMemsetAsync(a.bar, 0, sizeof(unsigned int), ctx->stream));
    void *args[] = {&a, &Y, &maxbits};
    GCK(cudaLaunchCooperativeKernel((const void *)k_tree_persist<T, R>, dim3(grid),
                                    dim3(threads), args, smem, ctx->stream));
    ctx->launches++;
}

struct SolveCall {
    grass_ctx_t ctx;
    grass_tree_t T;
    const TreeFactor *f;
    void *Y;
    unsigned long long *maxbits;
    grass_prec prec;
};

template <int R>
static void solve_R(const SolveCall &c) {
    if (c.prec == GRASS_FP64) solve_T<double, R>(c.ctx, c.T, *c.f, (double *)c.Y, c.maxbits);
    else solve_T<float, R>(c.ctx, c.T, *c.f, (float *)c.Y, c.maxbits);
}

void tree_solve_inplace(grass_ctx_t ctx, grass_tree_t T, const TreeFactor &f, int r,
                        grass_prec prec, void *Y, unsigned long long *maxbits) {
    const TreeSchedule &S = T->sched;
    const double s = prec == GRASS_FP64 ? 8.0 : 4.0, n = (double)T->g.n;
    const double bytes = 4.0 * n * r * s + S.n_rcv * (16.0 + 2.0 * s) +
                         (n - (double)T->nroots) * (16.0 + 4.0 * s);
    bool timed = ctx->t_begin(GRASS_KF_TREE, bytes);
    SolveCall c{ctx, T, &f, Y, maxbits, prec};
    GRASS_DISPATCH_R(r, solve_R, c);
    ctx->t_end(timed);
}

}  // namespace grass
