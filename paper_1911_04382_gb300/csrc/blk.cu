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

// Y = s * (L X + D .* X), (L X)_i = sum_j w_ij (X_i - X_j) (Eq. formula_laplacian).
// L lanes per row; each lane owns CPL chunks of the row and walks the row's
// entries in batches of B (indices and weights first, then the B gathers,
// then the sums), B chosen so that a lane has about 64 bytes of gathers in
// flight (more cost registers, and the occupancy lost outweighed the gain).
template <typename T, int R, int VB>
__global__ void __launch_bounds__(256) k_lapmm(int64_t n, const int32_t *__restrict__ ptr,
                                               const int32_t *__restrict__ col,
                                               const T *__restrict__ w, const T *__restrict__ D,
                                               const T *__restrict__ X, T *__restrict__ Y,
                                               const unsigned long long *scale_from,
                                               int32_t heavy_deg) {
    using RL = RowLay<T, R, VB>;
    constexpr int EL = RL::EL, L = RL::L, CPL = RL::CPL;
    // neighbours per batch: about 64 bytes of gathers in flight per lane
    constexpr int LB = CPL * EL * (int)sizeof(T);
    constexpr int B = LB >= 64 ? 1 : LB >= 32 ? 2 : 4;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t / L;
    if (i >= n) return;
    const int32_t j0 = __ldg(ptr + i), j1 = __ldg(ptr + i + 1);
    if (j1 - j0 > heavy_deg) return;      // a hub row: k_lapmm_heavy
    const int lane = (int)(t % L);
    const T s = (T)scale_of(scale_from);
    const int64_t off = lane * CPL * EL;   // first element of this lane in a row
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
            // past the row's end: reload its last entry (every address stays
            // inside the arrays) and mark the slot unused
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

template <typename T, int R, int VB>
static void lapmm_T(grass_ctx_t ctx, int64_t n, const int32_t *ptr, const int32_t *col,
                    const void *w, const void *D, const void *X, void *Y,
                    const unsigned long long *sf, const HeavyRows *hv) {
    constexpr int L = RowLay<T, R, VB>::L;
    const bool split = hv && hv->count > 0;
    launch(ctx, k_lapmm<T, R, VB>, cdiv(n * L, 256), 256, 0, n, ptr, col, (const T *)w,
           (const T *)D, (const T *)X, (T *)Y, sf, split ? (int32_t)kHeavyDeg : INT32_MAX);
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
    switch (chunk_bytes(R, sizeof(T), {X, Y})) {
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
// One edge per thread (no shuffles: the edge lists and the heats are read and
// written coalesced); a fixed grid walks the edges, each thread loading its
// next edge's endpoints and weight before it consumes this edge's row
// gathers, which it issues G chunks of 16 bytes per endpoint at a time.
// Every block ends with one atomicMax of its largest heat.
template <typename T, int R, int VB>
__global__ void __launch_bounds__(256) k_heat(int64_t moff, const int32_t *__restrict__ ou,
                                              const int32_t *__restrict__ ov,
                                              const T *__restrict__ ow, const T *__restrict__ H,
                                              const unsigned long long *scale_from,
                                              T *__restrict__ heat, unsigned long long *heatmax) {
    using RL = RowLay<T, R, VB>;
    constexpr int EL = RL::EL, C = R / EL;
    // chunks per endpoint in flight together: at most four, dividing the row
    constexpr int G = C % 4 == 0 ? 4 : C % 3 == 0 ? 3 : C % 2 == 0 ? 2 : 1;
    static_assert(C % G == 0, "chunk groups must tile the row");
    const T s = (T)scale_of(scale_from);
    const T s2 = s * s;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double mx = 0.0;
    int32_t eu = 0, ev = 0;
    T ew = (T)0;
    if (i < moff) {
        eu = __ldg(ou + i);
        ev = __ldg(ov + i);
        ew = __ldg(ow + i);
    }
    for (; i < moff; i += stride) {
        // the next edge of this thread (its last one reloads itself, so
        // every address stays inside the arrays)
        const int64_t inx = i + stride < moff ? i + stride : i;
        const int32_t nu = __ldg(ou + inx), nv = __ldg(ov + inx);
        const T nw = __ldg(ow + inx);
        const T *hu = H + (int64_t)eu * R;
        const T *hv = H + (int64_t)ev * R;
        T part = (T)0;
#pragma unroll
        for (int c0 = 0; c0 < C; c0 += G) {
            RowChunk<T, EL> a[G], b[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                a[g] = ld_row_chunk<T, EL>(hu + (c0 + g) * EL);
                b[g] = ld_row_chunk<T, EL>(hv + (c0 + g) * EL);
            }
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int e = 0; e < EL; ++e) {
                    const T d = a[g].v[e] - b[g].v[e];
                    part += d * d;
                }
        }
        const T h = ew * (part * s2);
        heat[i] = h;
        mx = fmax(mx, (double)h);
        eu = nu;
        ev = nv;
        ew = nw;
    }
    block_atomic_max(heatmax, mx);
}

template <typename T, int R, int VB>
static void heat_T(grass_ctx_t ctx, grass_sparsifier_t S, const void *H,
                   const unsigned long long *sf, void *heat, unsigned long long *hm) {
    const int64_t moff = S->m_off;
    const int sms = ctx->num_sms > 0 ? ctx->num_sms : 152;
    int nb = 0;
    GCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_heat<T, R, VB>, 256, 0));
    const int64_t grid = std::min<int64_t>(cdiv(moff, 256), (int64_t)sms * std::max(nb, 1));
    const T *ow = sizeof(T) == 8 ? (const T *)S->off_w64.p : (const T *)S->off_w32.p;
    launch(ctx, k_heat<T, R, VB>, grid, 256, 0, moff, (const int32_t *)S->off_u.p,
           (const int32_t *)S->off_v.p, ow, (const T *)H, sf, (T *)heat, hm);
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
