// blk.cu -- r-column kernels over the graph: Laplacian products (SpMM),
// Joule heat of the off-sparsifier edges, quadratic forms, power-of-two
// rescaling.
#include "common.cuh"

namespace grass {

__device__ inline double scale_of(const unsigned long long *scale_from) {
    return scale_from ? pow2_scale_from_bits(*scale_from) : 1.0;
}

// ---------------------------------------------------------------- row chunks
// The r values of a vertex are one contiguous row of r*sizeof(T) bytes.  The
// row kernels move it in chunks of VB bytes: 32 (256-bit loads of sm_100
// and later), 16 (float4 / double2), or single elements (VB = 0) -- the
// widest that divides the row and that the block's alignment allows; L
// consecutive lanes per row, CPL chunks a lane.  L divides 32, so a row
// never straddles a warp.
template <typename T, int R, int VB>
struct RowLay {
    static constexpr bool VEC = VB > 0 && (R * sizeof(T)) % VB == 0;
    static constexpr int EL = VEC ? int(VB / sizeof(T)) : 1;   // elements per chunk
    static constexpr int C = R / EL;                          // chunks per row
    static constexpr int L = (C % 8 == 0) ? 8 : (C % 4 == 0) ? 4 : (C % 2 == 0) ? 2 : 1;
    static constexpr int CPL = C / L;                         // chunks per lane
};

template <typename T, int EL>
struct RowChunk {
    T v[EL];
};

template <typename T, int EL>
__device__ __forceinline__ RowChunk<T, EL> ld_row_chunk(const T *p) {
    RowChunk<T, EL> c;
    if constexpr (sizeof(T) == 4 && EL == 8) {
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(c.v[0]), "=f"(c.v[1]), "=f"(c.v[2]), "=f"(c.v[3]), "=f"(c.v[4]), "=f"(c.v[5]),
              "=f"(c.v[6]), "=f"(c.v[7])
            : "l"(p));
    } else if constexpr (sizeof(T) == 8 && EL == 4) {
        asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
            : "=d"(c.v[0]), "=d"(c.v[1]), "=d"(c.v[2]), "=d"(c.v[3])
            : "l"(p));
    } else if constexpr (sizeof(T) == 4 && EL == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
        c.v[0] = q.x; c.v[1] = q.y; c.v[2] = q.z; c.v[3] = q.w;
    } else if constexpr (sizeof(T) == 8 && EL == 2) {
        const double2 q = __ldg(reinterpret_cast<const double2 *>(p));
        c.v[0] = q.x; c.v[1] = q.y;
    } else {
        static_assert(EL == 1, "chunk shape");
        c.v[0] = __ldg(p);
    }
    return c;
}

template <typename T, int EL>
__device__ __forceinline__ void st_row_chunk(T *p, const RowChunk<T, EL> &c) {
    if constexpr (sizeof(T) == 4 && EL == 8) {
        asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p),
                     "f"(c.v[0]), "f"(c.v[1]), "f"(c.v[2]), "f"(c.v[3]), "f"(c.v[4]), "f"(c.v[5]),
                     "f"(c.v[6]), "f"(c.v[7])
                     : "memory");
    } else if constexpr (sizeof(T) == 8 && EL == 4) {
        asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(c.v[0]), "d"(c.v[1]),
                     "d"(c.v[2]), "d"(c.v[3])
                     : "memory");
    } else if constexpr (sizeof(T) == 4 && EL == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(c.v[0], c.v[1], c.v[2], c.v[3]);
    } else if constexpr (sizeof(T) == 8 && EL == 2) {
        *reinterpret_cast<double2 *>(p) = make_double2(c.v[0], c.v[1]);
    } else {
        static_assert(EL == 1, "chunk shape");
        *p = c.v[0];
    }
}

inline bool aligned_to(const void *p, uintptr_t a) { return p == nullptr || ((uintptr_t)p & (a - 1)) == 0; }

// chunk width for r columns of `es`-byte elements over the given blocks
inline int chunk_bytes(int r, size_t es, std::initializer_list<const void *> blocks) {
    for (int vb : {32, 16}) {
        if ((r * es) % vb) continue;
        bool ok = true;
        for (const void *b : blocks) ok = ok && aligned_to(b, vb);
        if (ok) return vb;
    }
    return 0;
}

// The SpMM launch variant and chunk cap for (precision, r): the
// spmm_variant / spmm_chunk knobs when set (>= 0), else what the row-kernel
// autotuner kept (variant 0 and the widest chunk until it runs).
inline int r_slot(int r) {
    switch (r) {
        case 1: return 0;
        case 2: return 1;
        case 4: return 2;
        case 8: return 3;
        case 16: return 4;
        case 24: return 5;
        default: return 6;
    }
}
inline int spmm_variant_of(grass_ctx_t ctx, bool fp64, int r) {
    return ctx->spmm_variant >= 0 ? ctx->spmm_variant : ctx->spmm_tuned[fp64][r_slot(r)][1];
}
inline int spmm_chunk_of(grass_ctx_t ctx, bool fp64, int r) {
    return ctx->spmm_chunk >= 0 ? ctx->spmm_chunk : ctx->spmm_tuned[fp64][r_slot(r)][0];
}

// Y = s * (L X + D .* X), (L X)_i = sum_j w_ij (X_i - X_j) (Eq. formula_laplacian).
// L lanes per row; each lane owns CPL chunks of the row and walks the row's
// entries in batches of B (indices and weights first, then the B gathers,
// then the sums).  Launch variants (picked by the row-kernel autotuner, or
// the spmm_variant knob): B = BB, or by default sized so that a lane has
// about 64 bytes of gathers in flight; MB = the minimum resident blocks
// per SM asked of the compiler (a register cap); BLK = each block walks its
// own contiguous range of rows, 256 / L rows a step (the neighbour rows that
// earlier steps loaded are still in L1), else one row per L lanes of the
// grid.
template <typename T, int R, int VB, int BB, int MB, bool BLK>
__global__ void __launch_bounds__(256, MB) k_lapmm(int64_t n, const int32_t *__restrict__ ptr,
                                                   const int32_t *__restrict__ col,
                                                   const T *__restrict__ w, const T *__restrict__ D,
                                                   const T *__restrict__ X, T *__restrict__ Y,
                                                   const unsigned long long *scale_from,
                                                   int32_t heavy_deg) {
    using RL = RowLay<T, R, VB>;
    constexpr int EL = RL::EL, L = RL::L, CPL = RL::CPL;
    constexpr int LB = CPL * EL * (int)sizeof(T);
    constexpr int B = BB > 0 ? BB : LB >= 64 ? 1 : LB >= 32 ? 2 : 4;
    const int64_t per = BLK ? (n + gridDim.x - 1) / gridDim.x : 0;
    const int64_t lo = BLK ? min(n, (int64_t)blockIdx.x * per) : 0;
    const int64_t hi = BLK ? min(n, lo + per) : n;
    const int lane = (int)(threadIdx.x % L);
    const T s = (T)scale_of(scale_from);
    const int64_t off = lane * CPL * EL;   // first element of this lane in a row
    const int64_t step = BLK ? (int64_t)blockDim.x / L : n;
    for (int64_t i = BLK ? lo + threadIdx.x / L : ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / L;
         i < hi; i += step) {
        const int32_t j0 = __ldg(ptr + i), j1 = __ldg(ptr + i + 1);
        if (j1 - j0 > heavy_deg) continue;      // a hub row: k_lapmm_heavy
        RowChunk<T, EL> x0[CPL], acc[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            x0[c] = ld_row_chunk<T, EL>(X + i * R + off + c * EL);
#pragma unroll
            for (int e = 0; e < EL; ++e) acc[c].v[e] = (T)0;
        }
        for (int32_t j = j0; j < j1; j += B) {
            int32_t cj[B];
            T wj[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                // past the row's end: reload its last entry (every address
                // stays inside the arrays) and mark the slot unused
                const int32_t jb = j + b < j1 ? j + b : j1 - 1;
                cj[b] = __ldg(col + jb);
                wj[b] = __ldg(w + jb);
                if (j + b >= j1) cj[b] = -1;
            }
            RowChunk<T, EL> xq[B][CPL];
#pragma unroll
            for (int b = 0; b < B; ++b)
#pragma unroll
                for (int c = 0; c < CPL; ++c)
                    if (cj[b] >= 0) xq[b][c] = ld_row_chunk<T, EL>(X + (int64_t)cj[b] * R + off + c * EL);
#pragma unroll
            for (int b = 0; b < B; ++b)
                if (cj[b] >= 0)
#pragma unroll
                    for (int c = 0; c < CPL; ++c)
#pragma unroll
                        for (int e = 0; e < EL; ++e) acc[c].v[e] += wj[b] * (x0[c].v[e] - xq[b][c].v[e]);
        }
        if (D) {
            const T d = __ldg(D + i);
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < EL; ++e) acc[c].v[e] += d * x0[c].v[e];
        }
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
#pragma unroll
            for (int e = 0; e < EL; ++e) acc[c].v[e] *= s;
            st_row_chunk<T, EL>(Y + i * R + off + c * EL, acc[c]);
        }
    }
}

// The same product for the hub rows: one block of 256 threads per row, G =
// 256 / L groups of L lanes, group g taking the row's entries g, g + G, ...;
// the groups' partial sums meet in shared memory and are added in group
// order (deterministic), then D and the scale.
template <typename T, int R, int VB>
__global__ void __launch_bounds__(256) k_lapmm_heavy(const int32_t *__restrict__ rows,
                                                     const int32_t *__restrict__ ptr,
                                                     const int32_t *__restrict__ col,
                                                     const T *__restrict__ w,
                                                     const T *__restrict__ D,
                                                     const T *__restrict__ X, T *__restrict__ Y,
                                                     const unsigned long long *scale_from) {
    using RL = RowLay<T, R, VB>;
    constexpr int EL = RL::EL, L = RL::L, CPL = RL::CPL;
    constexpr int G = 256 / L;
    __shared__ T part[G * R];
    const int64_t i = rows[blockIdx.x];
    const int g = (int)threadIdx.x / L, lane = (int)threadIdx.x % L;
    const int64_t off = lane * CPL * EL;
    RowChunk<T, EL> x0[CPL], acc[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        x0[c] = ld_row_chunk<T, EL>(X + i * R + off + c * EL);
#pragma unroll
        for (int e = 0; e < EL; ++e) acc[c].v[e] = (T)0;
    }
    const int32_t j0 = __ldg(ptr + i), j1 = __ldg(ptr + i + 1);
    for (int32_t j = j0 + g; j < j1; j += G) {
        const int32_t cj = __ldg(col + j);
        const T wj = __ldg(w + j);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const RowChunk<T, EL> xq = ld_row_chunk<T, EL>(X + (int64_t)cj * R + off + c * EL);
#pragma unroll
            for (int e = 0; e < EL; ++e) acc[c].v[e] += wj * (x0[c].v[e] - xq.v[e]);
        }
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
        for (int e = 0; e < EL; ++e) part[g * R + off + c * EL + e] = acc[c].v[e];
    __syncthreads();
    const T s = (T)scale_of(scale_from);
    for (int q = (int)threadIdx.x; q < R; q += 256) {
        T y = (T)0;
        for (int k = 0; k < G; ++k) y += part[k * R + q];
        if (D) y += __ldg(D + i) * X[i * R + q];
        Y[i * R + q] = y * s;
    }
}

template <typename T, int R, int VB, int BB, int MB, bool BLK = false>
static void lapmm_V(grass_ctx_t ctx, int64_t n, const int32_t *ptr, const int32_t *col,
                    const void *w, const void *D, const void *X, void *Y,
                    const unsigned long long *sf, int32_t heavy_deg) {
    constexpr int L = RowLay<T, R, VB>::L;
    int64_t grid = cdiv(n * L, 256);
    if (BLK) {
        int nb = 0;
        GCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lapmm<T, R, VB, BB, MB, BLK>, 256, 0));
        const int sms = ctx->num_sms > 0 ? ctx->num_sms : 152;
        grid = std::min<int64_t>(grid, (int64_t)sms * std::max(nb, 1));
    }
    launch(ctx, k_lapmm<T, R, VB, BB, MB, BLK>, grid, 256, 0, n, ptr, col, (const T *)w,
           (const T *)D, (const T *)X, (T *)Y, sf, heavy_deg);
}

// The autotuned launch variants of the SpMM: (batch, minimum blocks per SM)
// = (rule, 1), (1, 1), (2, 1), (4, 1), (1, 6), (2, 6), and 6 / 7 = (rule, 1)
// / (1, 1) with each block on a contiguous range of rows.  Element-chunk
// layouts and r < 4 keep variant 0.
constexpr int kSpmmVariants = 8;

template <typename T, int R, int VB>
static void lapmm_T(grass_ctx_t ctx, int64_t n, const int32_t *ptr, const int32_t *col,
                    const void *w, const void *D, const void *X, void *Y,
                    const unsigned long long *sf, const HeavyRows *hv) {
    const bool split = hv && hv->count > 0;
    const int32_t hd = split ? (int32_t)kHeavyDeg : INT32_MAX;
    const int v = (VB == 0 || R < 4) ? 0 : spmm_variant_of(ctx, sizeof(T) == 8, R);
    switch (v) {
        case 1: lapmm_V<T, R, VB, 1, 1>(ctx, n, ptr, col, w, D, X, Y, sf, hd); break;
        case 2: lapmm_V<T, R, VB, 2, 1>(ctx, n, ptr, col, w, D, X, Y, sf, hd); break;
        case 3: lapmm_V<T, R, VB, 4, 1>(ctx, n, ptr, col, w, D, X, Y, sf, hd); break;
        case 4: lapmm_V<T, R, VB, 1, 6>(ctx, n, ptr, col, w, D, X, Y, sf, hd); break;
        case 5: lapmm_V<T, R, VB, 2, 6>(ctx, n, ptr, col, w, D, X, Y, sf, hd); break;
        case 6: lapmm_V<T, R, VB, 0, 1, true>(ctx, n, ptr, col, w, D, X, Y, sf, hd); break;
        case 7: lapmm_V<T, R, VB, 1, 1, true>(ctx, n, ptr, col, w, D, X, Y, sf, hd); break;
        default: lapmm_V<T, R, VB, 0, 1>(ctx, n, ptr, col, w, D, X, Y, sf, hd); break;
    }
    if (split)
        launch(ctx, k_lapmm_heavy<T, R, VB>, hv->count, 256, 0, (const int32_t *)hv->rows.p, ptr,
               col, (const T *)w, (const T *)D, (const T *)X, (T *)Y, sf);
}

template <typename T, int R>
static void lapmm_P(grass_ctx_t ctx, int64_t n, const int32_t *ptr, const int32_t *col,
                    const void *w, const void *D, const void *X, void *Y,
                    const unsigned long long *sf, const HeavyRows *hv) {
    // widest chunks that the row size and both blocks' alignment allow (a
    // caller's block or a slice of one may be only element-aligned)
    int vb = chunk_bytes(R, sizeof(T), {X, Y});
    if (vb == 32 && spmm_chunk_of(ctx, sizeof(T) == 8, R) == 16) vb = 16;
    switch (vb) {
        case 32: lapmm_T<T, R, 32>(ctx, n, ptr, col, w, D, X, Y, sf, hv); break;
        case 16: lapmm_T<T, R, 16>(ctx, n, ptr, col, w, D, X, Y, sf, hv); break;
        default: lapmm_T<T, R, 0>(ctx, n, ptr, col, w, D, X, Y, sf, hv); break;
    }
}

template <int R>
static void lapmm_R(grass_ctx_t ctx, grass_prec prec, int64_t n, const int32_t *ptr,
                    const int32_t *col, const void *w, const void *D, const void *X, void *Y,
                    const unsigned long long *sf, const HeavyRows *hv) {
    if (prec == GRASS_FP64) lapmm_P<double, R>(ctx, n, ptr, col, w, D, X, Y, sf, hv);
    else lapmm_P<float, R>(ctx, n, ptr, col, w, D, X, Y, sf, hv);
}

void lap_mm(grass_ctx_t ctx, int r, grass_prec prec, int64_t n, int64_t nnz, const int32_t *ptr,
            const int32_t *col, const void *w, const void *Dopt, const void *X, void *Y,
            const unsigned long long *scale_from, int fam, const HeavyRows *hv) {
    const double s = prec == GRASS_FP64 ? 8.0 : 4.0;
    const double bytes = 4.0 * (n + 1) + nnz * (4.0 + s) + 2.0 * n * r * s + (Dopt ? n * s : 0.0);
    // products with L_G over r > 1 columns are also a family of their own
    if (fam == GRASS_KF_SPMM_G && r > 1 && ctx->tfam == GRASS_KF_SPMM_BLK) fam = GRASS_KF_SPMM_BLK;
    bool timed = ctx->t_begin(fam, bytes);
    GRASS_DISPATCH_R(r, lapmm_R, ctx, prec, n, ptr, col, w, Dopt, X, Y, scale_from, hv);
    ctx->t_end(timed);
}

__global__ void k_heavy_list(int64_t n, const int32_t *ptr, int32_t deg, int64_t cap,
                             int32_t *rows, unsigned int *cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || ptr[i + 1] - ptr[i] <= deg) return;
    const unsigned int k = atomicAdd(cnt, 1u);
    if ((int64_t)k < cap) rows[k] = (int32_t)i;
}

void heavy_rows(grass_ctx_t ctx, int64_t n, int64_t nnz, const int32_t *ptr, HeavyRows &hv) {
    // at most nnz / (kHeavyDeg + 1) rows have more than kHeavyDeg entries
    const int64_t cap = nnz / (kHeavyDeg + 1) + 1;
    hv.rows.reserve(cap);
    hv.cnt.reserve(1);
    memset_d(ctx, hv.cnt.p, 0, sizeof(unsigned int));
    launch(ctx, k_heavy_list, cdiv(n, kBlock), kBlock, 0, n, ptr, (int32_t)kHeavyDeg, cap,
           hv.rows.p, hv.cnt.p);
    unsigned int c = 0;
    d2h(ctx, &c, hv.cnt.p, sizeof(c));
    hv.count = std::min<int64_t>(c, cap);
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
// P consecutive lanes per edge, each with C/P of the row's C
// chunks (P > 1: the P chunks of a row that one load instruction fetches
// lie in one cache line; partial sums meet by xor shuffles), E edges in
// flight per lane.  The edge lists and the heats are read and written in
// order; a fixed grid walks the edges, each lane loading its next edges'
// endpoints and weights before it consumes this step's row gathers.
// Every block ends with one atomicMax of its largest heat.
template <typename T, int R, int VB, int P, int E>
__global__ void __launch_bounds__(256) k_heat(int64_t moff, const int32_t *__restrict__ ou,
                                              const int32_t *__restrict__ ov,
                                              const T *__restrict__ ow, const T *__restrict__ H,
                                              const unsigned long long *scale_from,
                                              T *__restrict__ heat, unsigned long long *heatmax) {
    using RL = RowLay<T, R, VB>;
    constexpr int EL = RL::EL, C = R / EL;
    static_assert(P >= 1 && C % P == 0 && 32 % P == 0, "lanes must split the row");
    constexpr int CP = C / P;                 // chunks per lane
    // chunks per endpoint in flight together: at most four (two with two
    // edges in flight), dividing CP
    constexpr int GM = E == 1 ? 4 : 2;
    constexpr int G = CP % GM == 0 ? GM : (CP % 3 == 0 && GM >= 3) ? 3 : CP % 2 == 0 ? 2 : 1;
    static_assert(CP % G == 0, "chunk groups must tile the lane's share");
    const T s = (T)scale_of(scale_from);
    const T s2 = s * s;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = (int)(gt % P);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x / P;
    const int off = lane * CP * EL;
    double mx = 0.0;
    // E edges per lane and step: i, i + stride, ..., i + (E-1) stride; the
    // lane's edges beyond moff reload the last edge (every address stays
    // inside the arrays) and are not written
    int64_t i = gt / P;
    int32_t eu[E], ev[E];
    T ew[E];
    auto load_edges = [&](int64_t i0, int32_t (&u)[E], int32_t (&v)[E], T (&w)[E]) {
#pragma unroll
        for (int q = 0; q < E; ++q) {
            int64_t k = i0 + q * stride;
            if (k >= moff) k = moff - 1;
            u[q] = __ldg(ou + k);
            v[q] = __ldg(ov + k);
            w[q] = __ldg(ow + k);
        }
    };
    if (i < moff) load_edges(i, eu, ev, ew);
    // every lane of a group runs the same trip count (same i), so the
    // shuffles below see the whole group
    for (; i < moff; i += E * stride) {
        int32_t nu[E], nv[E];
        T nw[E];
        load_edges(i + E * stride < moff ? i + E * stride : i, nu, nv, nw);
        T part[E];
#pragma unroll
        for (int q = 0; q < E; ++q) part[q] = (T)0;
#pragma unroll
        for (int c0 = 0; c0 < CP; c0 += G) {
            RowChunk<T, EL> a[E][G], b[E][G];
#pragma unroll
            for (int q = 0; q < E; ++q)
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    a[q][g] = ld_row_chunk<T, EL>(H + (int64_t)eu[q] * R + off + (c0 + g) * EL);
                    b[q][g] = ld_row_chunk<T, EL>(H + (int64_t)ev[q] * R + off + (c0 + g) * EL);
                }
#pragma unroll
            for (int q = 0; q < E; ++q)
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int e = 0; e < EL; ++e) {
                        const T d = a[q][g].v[e] - b[q][g].v[e];
                        part[q] += d * d;
                    }
        }
#pragma unroll
        for (int q = 0; q < E; ++q) {
            if constexpr (P > 1) {
                const unsigned gm = ((1u << P) - 1u) << (((int)threadIdx.x & 31) & ~(P - 1));
#pragma unroll
                for (int d = P / 2; d > 0; d >>= 1) part[q] += __shfl_xor_sync(gm, part[q], d, P);
            }
            const int64_t k = i + q * stride;
            if (k < moff) {
                const T h = ew[q] * (part[q] * s2);
                if (lane == 0) heat[k] = h;
                mx = fmax(mx, (double)h);
            }
        }
#pragma unroll
        for (int q = 0; q < E; ++q) {
            eu[q] = nu[q];
            ev[q] = nv[q];
            ew[q] = nw[q];
        }
    }
    block_atomic_max(heatmax, mx);
}

// lanes per edge: the largest power of two (at most 4) dividing the row's
// chunks
template <typename T, int R, int VB>
struct HeatLanes {
    static constexpr int C = R / RowLay<T, R, VB>::EL;
    static constexpr int P = C % 4 == 0 ? 4 : C % 2 == 0 ? 2 : 1;
};

template <typename T, int R, int VB, int P, int E>
static void heat_L(grass_ctx_t ctx, grass_sparsifier_t S, const void *H,
                   const unsigned long long *sf, void *heat, unsigned long long *hm) {
    const int64_t moff = S->m_off;
    const int sms = ctx->num_sms > 0 ? ctx->num_sms : 152;
    int nb = 0;
    GCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_heat<T, R, VB, P, E>, 256, 0));
    const int64_t grid =
        std::min<int64_t>(cdiv(cdiv(moff, E) * P, 256), (int64_t)sms * std::max(nb, 1));
    const T *ow = sizeof(T) == 8 ? (const T *)S->off_w64.p : (const T *)S->off_w32.p;
    launch(ctx, k_heat<T, R, VB, P, E>, grid, 256, 0, moff, (const int32_t *)S->off_u.p,
           (const int32_t *)S->off_v.p, ow, (const T *)H, sf, (T *)heat, hm);
}

// heat_lanes knob / autotuner choice: 0 = P lanes per edge (by row size),
// one edge in flight; 1 = one lane per edge; 2 = P lanes, two edges in
// flight per lane; 3 = one lane, two edges
template <typename T, int R, int VB>
static void heat_T(grass_ctx_t ctx, grass_sparsifier_t S, const void *H,
                   const unsigned long long *sf, void *heat, unsigned long long *hm) {
    constexpr int P = HeatLanes<T, R, VB>::P;
    switch (ctx->heat_lanes) {
        case 1: heat_L<T, R, VB, 1, 1>(ctx, S, H, sf, heat, hm); break;
        case 2: heat_L<T, R, VB, P, 2>(ctx, S, H, sf, heat, hm); break;
        case 3: heat_L<T, R, VB, 1, 2>(ctx, S, H, sf, heat, hm); break;
        default: heat_L<T, R, VB, P, 1>(ctx, S, H, sf, heat, hm); break;
    }
}

template <typename T, int R>
static void heat_P(grass_ctx_t ctx, grass_sparsifier_t S, const void *H,
                   const unsigned long long *sf, void *heat, unsigned long long *hm) {
    switch (chunk_bytes(R, sizeof(T), {H})) {
        case 32: heat_T<T, R, 32>(ctx, S, H, sf, heat, hm); break;
        case 16: heat_T<T, R, 16>(ctx, S, H, sf, heat, hm); break;
        default: heat_T<T, R, 0>(ctx, S, H, sf, heat, hm); break;
    }
}

template <int R>
static void heat_R(grass_ctx_t ctx, grass_prec prec, grass_sparsifier_t S, const void *H,
                   const unsigned long long *sf, void *heat, unsigned long long *hm) {
    if (prec == GRASS_FP64) heat_P<double, R>(ctx, S, H, sf, heat, hm);
    else heat_P<float, R>(ctx, S, H, sf, heat, hm);
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

// ---------------------------------------------------------------- row-kernel autotuner

namespace grass {

// Times the r-column SpMM over the tree's graph under every launch variant
// and chunk width, and the heat kernel of the tree's off-tree edges in each
// of its forms; keeps the fastest on the context.  Results of either kernel
// are the same up to rounding order under any choice.
void autotune_rows(grass_ctx_t ctx, grass_tree_t T, int r, grass_prec prec, int32_t *best,
                   double *best_ms) {
    const GraphData &g = T->g;
    const int64_t n = g.n;
    const bool f64 = prec == GRASS_FP64;
    const size_t es = f64 ? 8 : 4;
    DBuf<char> X, Y;
    X.alloc(n * r * es);
    Y.alloc(n * r * es);
    memset_d(ctx, X.p, 0, n * r * es);
    const void *w = f64 ? (const void *)g.adj_w64.p : (const void *)g.adj_w32.p;
    cudaEvent_t e0, e1;
    GCK(cudaEventCreate(&e0));
    GCK(cudaEventCreate(&e1));
    const int keep_v = ctx->spmm_variant, keep_c = ctx->spmm_chunk, keep_h = ctx->heat_lanes;
    auto timed = [&](auto &&fn) {
        fn();   // warm
        GCK(cudaEventRecord(e0, ctx->stream));
        for (int k = 0; k < 5; ++k) fn();
        GCK(cudaEventRecord(e1, ctx->stream));
        GCK(cudaEventSynchronize(e1));
        float ms = 0.f;
        GCK(cudaEventElapsedTime(&ms, e0, e1));
        return ms / 5.0;
    };
    int bc = 0, bv = 0, bh = 0;
    double bms = 1e300, hms = 1e300;
    grass_sparsifier_t S = nullptr;
    try {
        const int widest = chunk_bytes(r, es, {X.p, Y.p});
        for (int cap : {0, 16}) {
            if (cap == 16 && widest != 32) continue;
            for (int v = 0; v < kSpmmVariants; ++v) {
                if (v > 0 && r < 4) break;
                ctx->spmm_chunk = cap;
                ctx->spmm_variant = v;
                const double ms = timed([&] {
                    lap_mm(ctx, r, prec, n, 2 * g.m, g.adj_ptr.p, g.adj_col.p, w, nullptr, X.p,
                           Y.p, nullptr, GRASS_KF_NONE, &g.heavy);
                });
                if (ms < bms) {
                    bms = ms;
                    bc = cap;
                    bv = v;
                }
            }
        }
        if (grass_sparsifier_create(ctx, T, &S) != GRASS_OK) fail(GRASS_ERR_CUDA, "autotune sparsifier");
        if (S->m_off > 0) {
            DBuf<char> heat;
            heat.alloc(S->m_off * es);
            unsigned long long *hm = (unsigned long long *)(ctx->scal.p + DS_MAX + 13);
            for (int h = 0; h <= 3; ++h) {
                ctx->heat_lanes = h;
                const double ms = timed([&] { heat_offs(ctx, r, prec, S, X.p, nullptr, heat.p, hm); });
                if (ms < hms) {
                    hms = ms;
                    bh = h;
                }
            }
        }
    } catch (...) {
        if (S) grass_sparsifier_destroy(S);
        ctx->spmm_variant = keep_v;
        ctx->spmm_chunk = keep_c;
        ctx->heat_lanes = keep_h;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    if (S) grass_sparsifier_destroy(S);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->spmm_variant = keep_v;
    ctx->spmm_chunk = keep_c;
    ctx->spmm_tuned[f64][r_slot(r)][0] = bc;
    ctx->spmm_tuned[f64][r_slot(r)][1] = bv;
    ctx->heat_lanes = bh;
    if (best) {
        best[0] = bc;
        best[1] = bv;
        best[2] = bh;
    }
    if (best_ms) {
        best_ms[0] = bms;
        best_ms[1] = hms < 1e299 ? hms : 0.0;
    }
}

}  // namespace grass
