// blk.cu -- r-column kernels over the graph: Laplacian products (SpMM),
// Joule heat of the off-sparsifier edges, quadratic forms, power-of-two
// rescaling.
#include "common.cuh"

namespace grass {

__device__ inline double scale_of(const unsigned long long *scale_from) {
    return scale_from ? pow2_scale_from_bits(*scale_from) : 1.0;
}

// Y = s * (L X + D .* X), (L X)_i = sum_j w_ij (X_i - X_j) (Eq. formula_laplacian).
template <typename T, int R>
__global__ void k_lapmm(int64_t n, const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                        const T *__restrict__ w, const T *__restrict__ D, const T *__restrict__ X,
                        T *__restrict__ Y, const unsigned long long *scale_from) {
    constexpr int TPR = Lay<R>::TPR, EPT = Lay<R>::EPT;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = t / TPR;
    if (i >= n) return;
    int c = (int)(t % TPR);
    const T s = (T)scale_of(scale_from);
    const T *xi = X + i * R + c * EPT;
    T x0[EPT], acc[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        x0[e] = xi[e];
        acc[e] = (T)0;
    }
    int32_t j1 = ptr[i + 1];
    for (int32_t j = ptr[i]; j < j1; ++j) {
        const T *xq = X + (int64_t)col[j] * R + c * EPT;
        T wj = w[j];
#pragma unroll
        for (int e = 0; e < EPT; ++e) acc[e] += wj * (x0[e] - xq[e]);
    }
    if (D) {
        T d = D[i];
#pragma unroll
        for (int e = 0; e < EPT; ++e) acc[e] += d * x0[e];
    }
    T *yi = Y + i * R + c * EPT;
#pragma unroll
    for (int e = 0; e < EPT; ++e) yi[e] = acc[e] * s;
}

template <int R>
static void lapmm_R(grass_ctx_t ctx, grass_prec prec, int64_t n, const int32_t *ptr,
                    const int32_t *col, const void *w, const void *D, const void *X, void *Y,
                    const unsigned long long *sf) {
    constexpr int TPR = Lay<R>::TPR;
    int64_t grid = cdiv(n * TPR, kBlock);
    if (prec == GRASS_FP64)
        launch(ctx, k_lapmm<double, R>, grid, kBlock, 0, n, ptr, col, (const double *)w,
               (const double *)D, (const double *)X, (double *)Y, sf);
    else
        launch(ctx, k_lapmm<float, R>, grid, kBlock, 0, n, ptr, col, (const float *)w,
               (const float *)D, (const float *)X, (float *)Y, sf);
}

void lap_mm(grass_ctx_t ctx, int r, grass_prec prec, int64_t n, int64_t nnz, const int32_t *ptr,
            const int32_t *col, const void *w, const void *Dopt, const void *X, void *Y,
            const unsigned long long *scale_from, int fam) {
    const double s = prec == GRASS_FP64 ? 8.0 : 4.0;
    const double bytes = 4.0 * (n + 1) + nnz * (4.0 + s) + 2.0 * n * r * s + (Dopt ? n * s : 0.0);
    bool timed = ctx->t_begin(fam, bytes);
    GRASS_DISPATCH_R(r, lapmm_R, ctx, prec, n, ptr, col, w, Dopt, X, Y, scale_from);
    ctx->t_end(timed);
}

// ---------------------------------------------------------------- conversions, scaling

template <typename T>
__global__ void k_convert(int64_t cnt, const double *src, T *dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) dst[i] = (T)src[i];
}

void convert_block(grass_ctx_t ctx, grass_prec prec, int64_t count, const double *src, void *dst) {
    if (prec == GRASS_FP64) copy_d(ctx, dst, src, count * sizeof(double));
    else launch(ctx, k_convert<float>, cdiv(count, kBlock), kBlock, 0, count, src, (float *)dst);
}

template <typename T>
__global__ void k_apply_pow2(int64_t cnt, T *X, const unsigned long long *sf) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) X[i] = X[i] * (T)pow2_scale_from_bits(*sf);
}

void apply_pow2(grass_ctx_t ctx, grass_prec prec, int64_t count, void *X,
                const unsigned long long *maxbits) {
    if (prec == GRASS_FP64)
        launch(ctx, k_apply_pow2<double>, cdiv(count, kBlock), kBlock, 0, count, (double *)X, maxbits);
    else
        launch(ctx, k_apply_pow2<float>, cdiv(count, kBlock), kBlock, 0, count, (float *)X, maxbits);
}

__device__ inline void warp_atomic_max(unsigned long long *maxbits, double v) {
    for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, d));
    if ((threadIdx.x & 31) == 0 && v > 0.0)
        atomicMax(maxbits, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__global__ void k_max_abs(int64_t cnt, const T *X, unsigned long long *maxbits) {
    double mx = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        mx = fmax(mx, fabs((double)X[i]));
    block_atomic_max(maxbits, mx);
}

void max_abs_bits(grass_ctx_t ctx, grass_prec prec, int64_t count, const void *X,
                  unsigned long long *maxbits) {
    int64_t grid = std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, cdiv(count, kBlock)));
    if (prec == GRASS_FP64)
        launch(ctx, k_max_abs<double>, grid, kBlock, 0, count, (const double *)X, maxbits);
    else
        launch(ctx, k_max_abs<float>, grid, kBlock, 0, count, (const float *)X, maxbits);
}

// ---------------------------------------------------------------- Joule heat
// heat_i = w_i * sum_j (H[u][j] - H[v][j])^2 for the i-th off-S edge
// (Eqs. formula_Joule, formula_pwr_iter5new, formula_pwr_iter6), with H
// multiplied by the pending power of two s (exact): heat = w s^2 sum(...).

template <typename T, int R>
__global__ void k_heat(int64_t moff, const int32_t *__restrict__ ou, const int32_t *__restrict__ ov,
                       const T *__restrict__ ow, const T *__restrict__ H,
                       const unsigned long long *scale_from, T *__restrict__ heat,
                       unsigned long long *heatmax) {
    constexpr int TPR = Lay<R>::TPR, EPT = Lay<R>::EPT;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = t / TPR;
    int c = (int)(t % TPR);
    T part = (T)0;
    if (i < moff) {
        const T *hu = H + (int64_t)ou[i] * R + c * EPT;
        const T *hv = H + (int64_t)ov[i] * R + c * EPT;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            T d = hu[e] - hv[e];
            part += d * d;
        }
    }
#pragma unroll
    for (int d = TPR / 2; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
    double hval = 0.0;
    if (i < moff && c == 0) {
        T s = (T)scale_of(scale_from);
        T h = ow[i] * (part * (s * s));
        heat[i] = h;
        hval = (double)h;
    }
    block_atomic_max(heatmax, hval);
}

template <int R>
static void heat_R(grass_ctx_t ctx, grass_prec prec, grass_sparsifier_t S, const void *H,
                   const unsigned long long *sf, void *heat, unsigned long long *hm) {
    constexpr int TPR = Lay<R>::TPR;
    int64_t moff = S->m_off;
    int64_t grid = cdiv(moff * TPR, kBlock);
    if (prec == GRASS_FP64)
        launch(ctx, k_heat<double, R>, grid, kBlock, 0, moff, (const int32_t *)S->off_u.p,
               (const int32_t *)S->off_v.p, (const double *)S->off_w64.p, (const double *)H, sf,
               (double *)heat, hm);
    else
        launch(ctx, k_heat<float, R>, grid, kBlock, 0, moff, (const int32_t *)S->off_u.p,
               (const int32_t *)S->off_v.p, (const float *)S->off_w32.p, (const float *)H, sf,
               (float *)heat, hm);
}

void heat_offs(grass_ctx_t ctx, int r, grass_prec prec, grass_sparsifier_t S, const void *H,
               const unsigned long long *scale_from, void *heat, unsigned long long *heatmax_bits) {
    memset_d(ctx, heatmax_bits, 0, sizeof(unsigned long long));
    const double s = prec == GRASS_FP64 ? 8.0 : 4.0;
    const double moff = (double)S->m_off, n = (double)S->tree->g.n;
    bool timed = ctx->t_begin(GRASS_KF_HEAT, moff * (8.0 + s) + n * r * s + moff * s);
    GRASS_DISPATCH_R(r, heat_R, ctx, prec, S, H, scale_from, heat, heatmax_bits);
    ctx->t_end(timed);
}

// ---------------------------------------------------------------- quadratic forms
// q[0] = x^T L_G x = sum_e w_e (x_u - x_v)^2, q[1] = same over S (Eq. 2);
// FP64 sums, fixed grid, per-block partials reduced in order by the last
// block.

template <typename T>
__global__ void k_quad(int64_t m, const int32_t *eu, const int32_t *ev, const double *ew,
                       const uint8_t *in_s, const T *x, double *partials, unsigned int *counter,
                       double *out) {
    __shared__ double shG[kBlock], shS[kBlock];
    __shared__ bool last;
    double g = 0.0, s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        double d = (double)x[eu[e]] - (double)x[ev[e]];
        double h = ew[e] * d * d;
        g += h;
        if (in_s[e]) s += h;
    }
    shG[threadIdx.x] = g;
    shS[threadIdx.x] = s;
    __syncthreads();
    for (int k = kBlock / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            shG[threadIdx.x] += shG[threadIdx.x + k];
            shS[threadIdx.x] += shS[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = shG[0];
        partials[2 * blockIdx.x + 1] = shS[0];
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x < 64) {
        // warp 0 sums qG, warp 1 qS: strided lanes, then a fixed xor tree
        __threadfence();
        const int lane = threadIdx.x & 31, which = threadIdx.x >> 5;
        double a = 0.0;
        for (unsigned k = lane; k < gridDim.x; k += 32) a += partials[2 * k + which];
        for (int d = 16; d > 0; d >>= 1) a += __shfl_xor_sync(0xffffffffu, a, d);
        if (lane == 0) out[which] = a;
        if (threadIdx.x == 0) *counter = 0u;
    }
}

void quad_forms(grass_ctx_t ctx, grass_prec prec, grass_sparsifier_t S, const void *x,
                double *out) {
    const GraphData &g = S->tree->g;
    int64_t grid = std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, cdiv(g.m, kBlock)));
    if (prec == GRASS_FP64)
        launch(ctx, k_quad<double>, grid, kBlock, 0, g.m, (const int32_t *)g.eu.p,
               (const int32_t *)g.ev.p, (const double *)g.ew64.p, (const uint8_t *)S->in_s.p,
               (const double *)x, ctx->partials.p, ctx->counters.p + 2, out);
    else
        launch(ctx, k_quad<float>, grid, kBlock, 0, g.m, (const int32_t *)g.eu.p,
               (const int32_t *)g.ev.p, (const double *)g.ew64.p, (const uint8_t *)S->in_s.p,
               (const float *)x, ctx->partials.p, ctx->counters.p + 2, out);
}

}  // namespace grass
