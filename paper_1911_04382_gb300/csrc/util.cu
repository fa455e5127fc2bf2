// util.cu -- prefix scans, deterministic column reductions, copies.
#include "common.cuh"

namespace grass {

// ---------------------------------------------------------------- copies

void d2h(grass_ctx_t ctx, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return;
    GCK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    ctx->sync();
}
void h2d(grass_ctx_t ctx, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return;
    GCK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    ctx->sync();
}
void memset_d(grass_ctx_t ctx, void *p, int v, size_t bytes) {
    if (bytes == 0) return;
    GCK(cudaMemsetAsync(p, v, bytes, ctx->stream));
}
void copy_d(grass_ctx_t ctx, void *dst, const void *src, size_t bytes) {
    if (bytes == 0 || dst == src) return;
    GCK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
}

// ---------------------------------------------------------------- scans
// Three-phase exclusive scan: per-tile sums, a single-block scan of the tile
// sums, then per-tile rescans with the tile offset.  Integer addition is
// associative, so the result does not depend on the tiling.

__device__ inline U64x2 operator+(U64x2 x, U64x2 y) { return U64x2{x.a + y.a, x.b + y.b}; }
__device__ inline U64x2 operator-(U64x2 x, U64x2 y) { return U64x2{x.a - y.a, x.b - y.b}; }

template <typename T>
__device__ inline T zero_of();
template <>
__device__ inline int64_t zero_of<int64_t>() { return 0; }
template <>
__device__ inline U64x2 zero_of<U64x2>() { return U64x2{0ull, 0ull}; }

__device__ inline int64_t shfl_up(int64_t v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ inline U64x2 shfl_up(U64x2 v, int d) {
    return U64x2{__shfl_up_sync(0xffffffffu, v.a, d), __shfl_up_sync(0xffffffffu, v.b, d)};
}

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// inclusive block scan of one value per thread; returns inclusive prefix,
// block total in *total.
template <typename T>
__device__ T block_incl_scan(T v, T *total) {
    __shared__ T warp_tot[kScanThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int d = 1; d < 32; d <<= 1) {
        T o = shfl_up(v, d);
        if (lane >= d) v = v + o;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        T w = lane < kScanThreads / 32 ? warp_tot[lane] : zero_of<T>();
        for (int d = 1; d < 32; d <<= 1) {
            T o = shfl_up(w, d);
            if (lane >= d) w = w + o;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    if (wid > 0) v = v + warp_tot[wid - 1];
    *total = warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
    return v;
}

template <typename T>
__global__ void k_tile_sums(const T *in, int64_t n, T *tsum) {
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    T acc = zero_of<T>();
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) acc = acc + in[i];
    }
    T tot;
    block_incl_scan(acc, &tot);
    if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_scan_tiles(T *tsum, int64_t ntiles) {
    // single block: exclusive scan of tile sums in chunks; tsum[ntiles] = total
    __shared__ T carry;
    if (threadIdx.x == 0) carry = zero_of<T>();
    __syncthreads();
    for (int64_t base = 0; base < ntiles; base += kScanThreads) {
        int64_t i = base + threadIdx.x;
        T v = i < ntiles ? tsum[i] : zero_of<T>();
        T tot;
        T inc = block_incl_scan(v, &tot);
        T c = carry;
        if (i < ntiles) tsum[i] = c + inc + zero_of<T>();   // inclusive for now
        __syncthreads();
        if (threadIdx.x == 0) carry = c + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) tsum[ntiles] = carry;
}

template <typename T>
__global__ void k_scan_apply(const T *in, T *out, int64_t n, const T *tincl, int64_t ntiles) {
    // each thread scans kScanItems consecutive elements of the tile
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T loc[kScanItems];
    T acc = zero_of<T>();
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        loc[k] = i < n ? in[i] : zero_of<T>();
        acc = acc + loc[k];
    }
    T tot;
    T inc = block_incl_scan(acc, &tot);
    T pre = (blockIdx.x == 0 ? zero_of<T>() : tincl[blockIdx.x - 1]) + (inc - acc);
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = pre;
        pre = pre + loc[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = tincl[ntiles];
}

template <typename T>
static void scan_impl(grass_ctx_t ctx, const T *in, T *out, int64_t n, T *total_host) {
    if (n <= 0) {
        GCK(cudaMemsetAsync(out, 0, sizeof(T), ctx->stream));
        if (total_host) d2h(ctx, total_host, out, sizeof(T));
        return;
    }
    int64_t ntiles = cdiv(n, kScanTile);
    T *tsum = ctx->scr<T>(SCR_SCAN, ntiles + 1);
    launch(ctx, k_tile_sums<T>, ntiles, kScanThreads, 0, in, n, tsum);
    launch(ctx, k_scan_tiles<T>, 1, kScanThreads, 0, tsum, ntiles);
    launch(ctx, k_scan_apply<T>, ntiles, kScanThreads, 0, in, out, n, (const T *)tsum, ntiles);
    if (total_host) d2h(ctx, total_host, out + n, sizeof(T));
}

void scan_i64(grass_ctx_t ctx, const int64_t *in, int64_t *out, int64_t n, int64_t *total_host) {
    scan_impl<int64_t>(ctx, in, out, n, total_host);
}
void scan_pair(grass_ctx_t ctx, const U64x2 *in, U64x2 *out, int64_t n, U64x2 *total_host) {
    scan_impl<U64x2>(ctx, in, out, n, total_host);
}

// ---------------------------------------------------------------- column dots
// Deterministic: a fixed grid; thread g accumulates the elements g, g+S,
// g+2S, ... of the flattened n*r block, S a multiple of r, so each thread
// stays in one column; per-block partials are reduced in a fixed order by
// the last block to finish.

template <typename T>
__global__ void k_dot_cols(int64_t total, int r, const T *A, const T *B, double *partials,
                           unsigned int *counter, double *out) {
    __shared__ double sh[kBlock];
    __shared__ bool last;
    int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    int64_t S = (nthreads / r) * r;
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (g < S)
        for (int64_t i = g; i < total; i += S) acc += (double)A[i] * (double)B[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    // per-column block sums: warp w reduces columns w, w+8, ...; lane l adds
    // the block's entries l, l+32, ... of that column, then a fixed xor tree
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t g0 = (int64_t)blockIdx.x * blockDim.x;
    for (int j = wid; j < r; j += nw) {
        double s = 0.0;
        for (int k = lane; k < kBlock; k += 32) {
            int64_t gk = g0 + k;
            if (gk < S && (int)(gk % r) == j) s += sh[k];
        }
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) {
            partials[(int64_t)j * gridDim.x + blockIdx.x] = s;
            __threadfence();
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) {
        __threadfence();
        for (int j = wid; j < r; j += nw) {
            double s = 0.0;
            for (unsigned b = lane; b < gridDim.x; b += 32) s += partials[(int64_t)j * gridDim.x + b];
            for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
            if (lane == 0) out[j] = s;
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
}

void dot_cols(grass_ctx_t ctx, int r, grass_prec prec, int64_t n, const void *A, const void *B,
              double *out) {
    int64_t total = n * r;
    int64_t grid = std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, cdiv(total, kBlock)));
    if (prec == GRASS_FP64)
        launch(ctx, k_dot_cols<double>, grid, kBlock, 0, total, r, (const double *)A,
               (const double *)B, ctx->partials.p, ctx->counters.p, out);
    else
        launch(ctx, k_dot_cols<float>, grid, kBlock, 0, total, r, (const float *)A,
               (const float *)B, ctx->partials.p, ctx->counters.p + 1, out);
}

__global__ void k_ones64(int64_t n, double *o) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = 1.0;
}

__global__ void k_sub_mean(int64_t n, double *v, const double *sum) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] -= *sum / (double)n;
}

void project_ones(grass_ctx_t ctx, int64_t n, double *v) {
    double *ones = ctx->scr<double>(SCR_ONES, n);
    double *sum = ctx->scal.p + DS_RED + 60;
    launch(ctx, k_ones64, cdiv(n, kBlock), kBlock, 0, n, ones);
    dot_cols(ctx, 1, GRASS_FP64, n, v, ones, sum);
    launch(ctx, k_sub_mean, cdiv(n, kBlock), kBlock, 0, n, v, (const double *)sum);
}

}  // namespace grass
