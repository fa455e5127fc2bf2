// tree_solve.cuh -- device code of the tree solve, shared by the stand-alone
// solve kernel (solve.cu) and the fused CG kernel (krylov.cu).
//
// Forward elimination: round by round, every vertex that receives updates
// adds m * y_v for each neighbour v eliminated in that round.  Backward
// substitution: rounds in reverse, x_v = y_v / d_v + (w1/d_v) x_n1 +
// (w2/d_v) x_n2.  The big first rounds run across the whole grid, separated
// by bounded grid barriers; the small last rounds run in block 0 on the
// surviving vertices staged in shared memory.  Each item is one packed
// 16-byte record plus its coefficients, and every thread loads its first
// record of the next round before waiting at the barrier.
#pragma once

#include "common.cuh"

namespace grass {

template <typename T>
struct PackT;
template <>
struct PackT<float> {
    using V2 = float2;
    using V4 = float4;
};
template <>
struct PackT<double> {
    using V2 = double2;
    using V4 = Dbl4;
};

template <typename T>
struct TreeKArgs {
    int rounds, K1;
    int64_t base, ntl, r0, e0, c0;
    // the tail (rounds K1..): first forward record and count, first backward
    // record and count, first contribution index and count
    int64_t tf0, tnf, tg0, tnb, tc0, ntc;
    const int64_t *rcv_off, *elim_off;
    const int4 *fwd_rec, *bwd_rec, *fwd_loc, *bwd_loc;
    const typename PackT<T>::V2 *fm;
    const typename PackT<T>::V4 *bc;
    const int32_t *beg, *cv, *tail_vid, *contrib_loc;
    const T *cm;
    const T *root_invd;   // [nroots], roots in tail order
    int nroots;
    unsigned int *bar;
    long long budget;
    int *err;
};

template <typename T, int R>
__device__ inline void fwd_packed(int64_t i, int c, int4 r, typename PackT<T>::V2 mm,
                                  const int32_t *beg, const int32_t *cv, const T *cm, T *Y) {
    constexpr int EPT = Lay<R>::EPT;
    T *yu = Y + (int64_t)r.x * R + c * EPT;
    const T *y0 = Y + (int64_t)r.y * R + c * EPT;
    T acc[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) acc[e] = yu[e] + mm.x * y0[e];
    if (r.z >= 0) {
        const T *y1 = Y + (int64_t)r.z * R + c * EPT;
#pragma unroll
        for (int e = 0; e < EPT; ++e) acc[e] += mm.y * y1[e];
    }
    if (r.w >= 0) {
        for (int32_t k = r.w; k < beg[i + 1]; ++k) {
            const T *yv = Y + (int64_t)cv[k] * R + c * EPT;
            T mlt = cm[k];
#pragma unroll
            for (int e = 0; e < EPT; ++e) acc[e] += mlt * yv[e];
        }
    }
#pragma unroll
    for (int e = 0; e < EPT; ++e) yu[e] = acc[e];
}

template <typename T, int R>
__device__ inline double bwd_packed(int c, int4 r, typename PackT<T>::V4 cf, T *Y) {
    constexpr int EPT = Lay<R>::EPT;
    T *yv = Y + (int64_t)r.x * R + c * EPT;
    const T *xa = Y + (int64_t)r.y * R + c * EPT;
    T x[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) x[e] = cf.x * yv[e] + cf.y * xa[e];
    if (r.z >= 0) {
        const T *xb = Y + (int64_t)r.z * R + c * EPT;
#pragma unroll
        for (int e = 0; e < EPT; ++e) x[e] += cf.z * xb[e];
    }
    double mx = 0.0;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        yv[e] = x[e];
        mx = fmax(mx, fabs((double)x[e]));
    }
    return mx;
}

// A thread's items of one round, at most kBatch of them, loaded together so
// their latencies overlap: item j is index lo + slot + j * nslots.  More
// than one item per batch spills, at 64 registers a thread (1024 threads)
// and inside the fused Krylov kernels at 128.
constexpr int kBatch = 1;

template <typename T>
struct FwdBatch {
    int4 r[kBatch];
    typename PackT<T>::V2 m[kBatch];
    int64_t i0, step;   // item j is i0 + j * step
    int cnt;
};

template <typename T>
struct BwdBatch {
    int4 r[kBatch];
    typename PackT<T>::V4 c[kBatch];
    int cnt;
};

// Item i of a round: record rec[i - off0] and coefficients cf[i - off0]
// (global arrays with off0 = 0, or the tail's shared-memory copies indexed
// from the tail's first item).
template <typename T>
__device__ __forceinline__ void load_fwd(FwdBatch<T> &b, const int4 *rec,
                                         const typename PackT<T>::V2 *cf, int64_t off0, int64_t lo,
                                         int64_t hi, int64_t slot, int64_t nslots) {
    b.cnt = 0;
    b.i0 = lo + slot;
    b.step = nslots;
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
        int64_t i = lo + slot + j * nslots;
        if (i < hi) {
            b.r[j] = rec[i - off0];
            b.m[j] = cf[i - off0];
            b.cnt = j + 1;
        }
    }
}

template <typename T>
__device__ __forceinline__ void load_bwd(BwdBatch<T> &b, const int4 *rec,
                                         const typename PackT<T>::V4 *cf, int64_t off0, int64_t lo,
                                         int64_t hi, int64_t slot, int64_t nslots) {
    b.cnt = 0;
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
        int64_t p = lo + slot + j * nslots;
        if (p < hi) {
            b.r[j] = rec[p - off0];
            b.c[j] = cf[p - off0];
            b.cnt = j + 1;
        }
    }
}

// Shared-memory layout of the tail: the staged rows (ntl x R values), then
// its forward and backward records and coefficients, then its contribution
// lists beyond the two inline ones (ends per record, contributor local ids,
// multipliers), each 32-byte aligned.  Everything after the rows depends on
// the tree alone: staged once per launch (tree_tail_stage).
template <typename T, int R>
struct TailSmem {
    int4 *frec, *brec;
    typename PackT<T>::V2 *fm;
    typename PackT<T>::V4 *bc;
    int32_t *cend, *cloc;
    T *cmul;
    __device__ TailSmem(T *ys, int64_t ntl, int64_t nf, int64_t nb, int64_t nc) {
        auto up = [](size_t x) { return (x + 31) & ~size_t(31); };
        char *p = reinterpret_cast<char *>(ys);
        size_t o = up((size_t)ntl * R * sizeof(T));
        frec = reinterpret_cast<int4 *>(p + o);
        o = up(o + (size_t)nf * sizeof(int4));
        brec = reinterpret_cast<int4 *>(p + o);
        o = up(o + (size_t)nb * sizeof(int4));
        fm = reinterpret_cast<typename PackT<T>::V2 *>(p + o);
        o = up(o + (size_t)nf * sizeof(typename PackT<T>::V2));
        bc = reinterpret_cast<typename PackT<T>::V4 *>(p + o);
        o = up(o + (size_t)nb * sizeof(typename PackT<T>::V4));
        cend = reinterpret_cast<int32_t *>(p + o);
        o = up(o + (size_t)nf * sizeof(int32_t));
        cloc = reinterpret_cast<int32_t *>(p + o);
        o = up(o + (size_t)nc * sizeof(int32_t));
        cmul = reinterpret_cast<T *>(p + o);
    }
    // bytes of the whole layout (host and device)
    __host__ __device__ static size_t bytes(int64_t ntl, int64_t nf, int64_t nb, int64_t nc) {
        auto up = [](size_t x) { return (x + 31) & ~size_t(31); };
        size_t o = up((size_t)ntl * R * sizeof(T));
        o = up(o + (size_t)nf * sizeof(int4));
        o = up(o + (size_t)nb * sizeof(int4));
        o = up(o + (size_t)nf * sizeof(typename PackT<T>::V2));
        o = up(o + (size_t)nb * sizeof(typename PackT<T>::V4));
        o = up(o + (size_t)nf * sizeof(int32_t));
        o = up(o + (size_t)nc * sizeof(int32_t));
        return o + (size_t)nc * sizeof(T);
    }
};

// Forward items of a batch on the vector V (global Y, or the tail's shared
// copy with ids shifted by `base`); all gathers issued before any store.  On
// the global vector the end of a record's contribution list and its first
// contributor and multiplier load with the inline gathers, so a receiver
// with more than two contributions costs one more round trip, not three.
template <typename T, int R>
__device__ __forceinline__ void run_fwd(const FwdBatch<T> &b, const TreeKArgs<T> &a, T *V, int64_t base,
                               const TailSmem<T, R> *sm, int c) {
    constexpr int EPT = Lay<R>::EPT;
    T yu[kBatch][EPT], y0[kBatch][EPT], y1[kBatch][EPT];
    int32_t kend[kBatch], v3[kBatch];
    T m3[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
        if (j >= b.cnt) break;
        const int4 r = b.r[j];
        if (!sm && r.w >= 0) {
            kend[j] = a.beg[b.i0 + j * b.step + 1];
            v3[j] = a.cv[r.w];
            m3[j] = a.cm[r.w];
        }
        const T *pu = V + (r.x - base) * R + c * EPT;
        const T *p0 = V + (r.y - base) * R + c * EPT;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            yu[j][e] = pu[e];
            y0[j][e] = p0[e];
            y1[j][e] = (T)0;
        }
        if (r.z >= 0) {
            const T *p1 = V + (r.z - base) * R + c * EPT;
#pragma unroll
            for (int e = 0; e < EPT; ++e) y1[j][e] = p1[e];
        }
    }
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
        if (j >= b.cnt) break;
        const int4 r = b.r[j];
        const auto mm = b.m[j];
        T acc[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) acc[e] = yu[j][e] + mm.x * y0[j][e];
        if (r.z >= 0) {
#pragma unroll
            for (int e = 0; e < EPT; ++e) acc[e] += mm.y * y1[j][e];
        }
        if (r.w >= 0) {
            const int64_t i = b.i0 + j * b.step;
            if (sm) {
                // tail: shared copies, indexed from the tail's first record
                // and first contribution
                for (int64_t k = r.w - a.tc0; k < sm->cend[i - a.tf0]; ++k) {
                    const T *pv = V + ((int64_t)sm->cloc[k] - base) * R + c * EPT;
                    const T mlt = sm->cmul[k];
#pragma unroll
                    for (int e = 0; e < EPT; ++e) acc[e] += mlt * pv[e];
                }
            } else {
                const T *p3 = V + ((int64_t)v3[j] - base) * R + c * EPT;
#pragma unroll
                for (int e = 0; e < EPT; ++e) acc[e] += m3[j] * p3[e];
                for (int32_t k = r.w + 1; k < kend[j]; ++k) {
                    const T *pv = V + ((int64_t)a.cv[k] - base) * R + c * EPT;
                    const T mlt = a.cm[k];
#pragma unroll
                    for (int e = 0; e < EPT; ++e) acc[e] += mlt * pv[e];
                }
            }
        }
        T *pu = V + (r.x - base) * R + c * EPT;
#pragma unroll
        for (int e = 0; e < EPT; ++e) pu[e] = acc[e];
    }
}

// Returns max |x| over the values written (in T's precision; 0 unless TRACK).
template <typename T, int R, bool TRACK = true>
__device__ __forceinline__ double run_bwd(const BwdBatch<T> &b, T *V, int64_t base, int c) {
    constexpr int EPT = Lay<R>::EPT;
    T yv[kBatch][EPT], xa[kBatch][EPT], xb[kBatch][EPT];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
        if (j >= b.cnt) break;
        const int4 r = b.r[j];
        const T *pv = V + (r.x - base) * R + c * EPT;
        const T *pa = V + (r.y - base) * R + c * EPT;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            yv[j][e] = pv[e];
            xa[j][e] = pa[e];
            xb[j][e] = (T)0;
        }
        if (r.z >= 0) {
            const T *pb = V + (r.z - base) * R + c * EPT;
#pragma unroll
            for (int e = 0; e < EPT; ++e) xb[j][e] = pb[e];
        }
    }
    T mx = (T)0;
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
        if (j >= b.cnt) break;
        const int4 r = b.r[j];
        const auto cf = b.c[j];
        T *pv = V + (r.x - base) * R + c * EPT;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            T x = cf.x * yv[j][e] + cf.y * xa[j][e];
            if (r.z >= 0) x += cf.z * xb[j][e];
            pv[e] = x;
            if (TRACK) mx = fmax(mx, fabs(x));
        }
    }
    return (double)mx;
}

// Block 0 copies the tail's records, coefficients and contribution lists
// into shared memory (after the rows); once per launch, before the first
// solve (the solve's tail waits on __syncthreads after it).
template <typename T, int R>
__device__ inline void tree_tail_stage(const TreeKArgs<T> &a, T *ys) {
    if (blockIdx.x != 0 || a.K1 >= a.rounds) return;
    const TailSmem<T, R> sm(ys, a.ntl, a.tnf, a.tnb, a.ntc);
    for (int64_t i = threadIdx.x; i < a.tnf; i += blockDim.x) {
        sm.frec[i] = a.fwd_loc[a.tf0 - a.r0 + i];
        sm.fm[i] = a.fm[a.tf0 + i];
        sm.cend[i] = (int32_t)(a.beg[a.tf0 + i + 1] - a.tc0);
    }
    for (int64_t i = threadIdx.x; i < a.tnb; i += blockDim.x) {
        sm.brec[i] = a.bwd_loc[a.tg0 - a.e0 + i];
        sm.bc[i] = a.bc[a.tg0 + i];
    }
    for (int64_t k = threadIdx.x; k < a.ntc; k += blockDim.x) {
        sm.cloc[k] = a.contrib_loc[a.tc0 - a.c0 + k];
        sm.cmul[k] = a.cm[a.tc0 + k];
    }
}

// Solve in place on Y (n x R).  Called by every thread of a cooperative
// grid; returns false when a barrier wait ran out (the caller must return).
// mx accumulates max |x| over the values this thread wrote.  Ends without
// a trailing grid barrier.
template <typename T, int R, bool TRACK = true>
__device__ __forceinline__ bool tree_solve_dev(const TreeKArgs<T> &a, T *Y, unsigned int &epoch,
                                      double &mx, T *ys) {
    constexpr int TPR = Lay<R>::TPR;
    __shared__ int64_t s_roff[kMaxRounds + 1], s_eoff[kMaxRounds + 1];
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = (int)(gt % TPR);
    const int64_t slot = gt / TPR;
    const int64_t nslots = (int64_t)gridDim.x * blockDim.x / TPR;
    __syncthreads();
    for (int k = threadIdx.x; k <= a.rounds; k += blockDim.x) {
        s_roff[k] = a.rcv_off[k];
        s_eoff[k] = a.elim_off[k];
    }
    __syncthreads();
    // rounds 0 .. K1-1 forward across the grid; the next round's batch is
    // loaded before the barrier
    FwdBatch<T> fb;
    fb.cnt = 0;
    if (a.K1 > 0) load_fwd(fb, a.fwd_rec, a.fm, 0, s_roff[0], s_roff[1], slot, nslots);
    for (int k = 0; k < a.K1; ++k) {
        run_fwd<T, R>(fb, a, Y, 0, (const TailSmem<T, R> *)nullptr, c);
        for (int64_t lo = s_roff[k] + kBatch * nslots; lo < s_roff[k + 1]; lo += kBatch * nslots) {
            FwdBatch<T> more;
            load_fwd(more, a.fwd_rec, a.fm, 0, lo, s_roff[k + 1], slot, nslots);
            run_fwd<T, R>(more, a, Y, 0, (const TailSmem<T, R> *)nullptr, c);
        }
        if (k + 1 < a.K1) load_fwd(fb, a.fwd_rec, a.fm, 0, s_roff[k + 1], s_roff[k + 2], slot, nslots);
        if (!grid_sync(a.bar, a.budget, a.err, epoch)) return false;
    }
    // rounds K1 .. end in block 0, on the tail vertices gathered into shared
    // memory; the tail's records, coefficients and contribution lists are
    // there already (tree_tail_stage), so each round runs from shared memory
    if (blockIdx.x == 0) {
        const int64_t bslot = threadIdx.x / TPR, bslots = blockDim.x / TPR;
        const int64_t base = a.base, ntl = a.ntl;
        const int64_t f0 = a.tf0, g0 = a.tg0;
        const TailSmem<T, R> sm(ys, ntl, a.tnf, a.tnb, a.ntc);
        for (int64_t idx = threadIdx.x; idx < ntl * R; idx += blockDim.x)
            ys[idx] = Y[(int64_t)a.tail_vid[base + idx / R] * R + idx % R];
        __syncthreads();
        FwdBatch<T> tb;
        tb.cnt = 0;
        if (a.K1 < a.rounds)
            load_fwd(tb, sm.frec, sm.fm, f0, s_roff[a.K1], s_roff[a.K1 + 1], bslot, bslots);
        for (int k = a.K1; k < a.rounds; ++k) {
            run_fwd<T, R>(tb, a, ys, base, &sm, c);
            for (int64_t lo = s_roff[k] + kBatch * bslots; lo < s_roff[k + 1]; lo += kBatch * bslots) {
                FwdBatch<T> more;
                load_fwd(more, sm.frec, sm.fm, f0, lo, s_roff[k + 1], bslot, bslots);
                run_fwd<T, R>(more, a, ys, base, &sm, c);
            }
            if (k + 1 < a.rounds)
                load_fwd(tb, sm.frec, sm.fm, f0, s_roff[k + 1], s_roff[k + 2], bslot, bslots);
            __syncthreads();
        }
        BwdBatch<T> bb;
        bb.cnt = 0;
        if (a.K1 < a.rounds)
            load_bwd(bb, sm.brec, sm.bc, g0, s_eoff[a.rounds - 1], s_eoff[a.rounds], bslot, bslots);
        for (int64_t q = bslot; q < a.nroots; q += bslots) {
            constexpr int EPT = Lay<R>::EPT;
            T *yr = ys + (ntl - a.nroots + q) * R + c * EPT;   // the roots come last
            const T ri = a.root_invd[q];
#pragma unroll
            for (int e = 0; e < EPT; ++e) yr[e] = ri * yr[e];
        }
        __syncthreads();
        for (int k = a.rounds - 1; k >= a.K1; --k) {
            run_bwd<T, R, false>(bb, ys, base, c);
            for (int64_t lo = s_eoff[k] + kBatch * bslots; lo < s_eoff[k + 1]; lo += kBatch * bslots) {
                BwdBatch<T> more;
                load_bwd(more, sm.brec, sm.bc, g0, lo, s_eoff[k + 1], bslot, bslots);
                run_bwd<T, R, false>(more, ys, base, c);
            }
            if (k - 1 >= a.K1)
                load_bwd(bb, sm.brec, sm.bc, g0, s_eoff[k - 1], s_eoff[k], bslot, bslots);
            __syncthreads();
        }
        T tm = (T)0;
        for (int64_t idx = threadIdx.x; idx < ntl * R; idx += blockDim.x) {
            T v = ys[idx];
            Y[(int64_t)a.tail_vid[base + idx / R] * R + idx % R] = v;
            if (TRACK) tm = fmax(tm, fabs(v));
        }
        if (TRACK) mx = fmax(mx, (double)tm);
    }
    // rounds K1-1 .. 0 backward across the grid
    BwdBatch<T> gb;
    gb.cnt = 0;
    if (a.K1 > 0) load_bwd(gb, a.bwd_rec, a.bc, 0, s_eoff[a.K1 - 1], s_eoff[a.K1], slot, nslots);
    if (a.K1 > 0 && !grid_sync(a.bar, a.budget, a.err, epoch)) return false;
    for (int k = a.K1 - 1; k >= 0; --k) {
        if (TRACK) mx = fmax(mx, run_bwd<T, R, TRACK>(gb, Y, 0, c));
        else run_bwd<T, R, false>(gb, Y, 0, c);
        for (int64_t lo = s_eoff[k] + kBatch * nslots; lo < s_eoff[k + 1]; lo += kBatch * nslots) {
            BwdBatch<T> more;
            load_bwd(more, a.bwd_rec, a.bc, 0, lo, s_eoff[k + 1], slot, nslots);
            if (TRACK) mx = fmax(mx, run_bwd<T, R, TRACK>(more, Y, 0, c));
            else run_bwd<T, R, false>(more, Y, 0, c);
        }
        if (k > 0) {
            load_bwd(gb, a.bwd_rec, a.bc, 0, s_eoff[k - 1], s_eoff[k], slot, nslots);
            if (!grid_sync(a.bar, a.budget, a.err, epoch)) return false;
        }
    }
    return true;
}

// One-column element loops.  FP32 vectors are walked in 16-byte chunks:
// thread gt takes chunks gt, gt + nth, ... (four floats, one vector access
// per operand) and the n mod 4 leftover elements go to threads 0, 1, 2.
// Every such loop over the same vectors uses this mapping, so an element is
// always read and written by the same thread.  FP64 vectors (which may be
// the caller's own, 8-byte aligned) take one element per step.
template <typename T>
struct Chunk {
    static constexpr int W = sizeof(T) == 4 ? 4 : 1;
};

template <typename T, typename F>
__device__ __forceinline__ void for_chunks(int64_t n, int64_t gt, int64_t nth, F &&f) {
    constexpr int W = Chunk<T>::W;
    const int64_t nv = n / W;
    for (int64_t v = gt; v < nv; v += nth) f(v * W, W);
    if constexpr (W > 1) {
        if (gt < n - nv * W) f(nv * W + gt, 1);
    }
}

template <typename T>
__device__ __forceinline__ void ld_chunk(const T *p, int cnt, T (&v)[Chunk<T>::W]) {
    if constexpr (Chunk<T>::W == 4) {
        if (cnt == 4) {
            const float4 q = *reinterpret_cast<const float4 *>(p);
            v[0] = q.x;
            v[1] = q.y;
            v[2] = q.z;
            v[3] = q.w;
            return;
        }
        v[1] = v[2] = v[3] = (T)0;
    }
    v[0] = p[0];
}

template <typename T>
__device__ __forceinline__ void st_chunk(T *p, int cnt, const T (&v)[Chunk<T>::W]) {
    if constexpr (Chunk<T>::W == 4) {
        if (cnt == 4) {
            *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
            return;
        }
    }
    p[0] = v[0];
}

// ---------------------------------------------------------------- scan form (D = 0, r = 1)
// Grounded solve of L_T x = b along the Euler tour (euler.cu): with S the
// exclusive prefix sums of b placed at the tour's entries, the current up
// v's parent edge is c_v = (S[out(v)] - S[in(v)]) / w_v; with S2 the prefix
// sums of +c at entries and -c at exits, x_v = S2 up to and including
// in(v).  The same in the tree's preorder over the n vertex slots
// (euler_solve_pre).  FP64 (or float-pair) sums; each block scans a
// contiguous stretch and every block derives the stretch offsets from the
// per-block totals in one fixed order, so the result does not depend on
// timing.

struct EulerKArgs {
    int64_t L, n;
    const int32_t *tour, *ein, *eout;
    const uint8_t *head;    // [L] 1 at the first position of every tree's tour
    // preorder form (pre = 1): the vectors are in the tree's preorder;
    // head_n [n] marks every tree's root slot, D [n] holds step 2's values
    int pre;
    const uint8_t *head_n;
    void *D;
    const void *ipw;        // [n] 1 / weight of v's parent edge (T)
    void *S, *C;            // [L] prefix sums (SumOf<T>), [n] currents (T)
    double *part;           // [6 * gridDim.x]: block pairs and first heads
};

constexpr int kEulerMaxGrid = 2048;

// Prefix sums of the scan form.  Double vectors: FP64.  Float vectors: a
// float pair (sum and error, two-sum on every add), about 44 significant
// bits, enough for the subtree sums taken as differences of prefix sums,
// with no FP64 arithmetic per tour position.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, e);
    return DF{hi, __fsub_rn(e, __fsub_rn(hi, s))};
}
template <typename T>
struct SumOf {
    using type = double;
};
template <>
struct SumOf<float> {
    using type = DF;
};
__device__ __forceinline__ double s_add(double a, double b) { return a + b; }
__device__ __forceinline__ DF s_add(DF a, DF b) { return df_add(a, b); }
__device__ __forceinline__ double s_sub(double a, double b) { return a - b; }
__device__ __forceinline__ DF s_sub(DF a, DF b) { return df_add(a, DF{-b.hi, -b.lo}); }
template <typename V>
__device__ __forceinline__ V s_from(double x);
template <>
__device__ __forceinline__ double s_from<double>(double x) { return x; }
template <>
__device__ __forceinline__ DF s_from<DF>(double x) {
    const float h = (float)x;
    return DF{h, (float)(x - (double)h)};
}
__device__ __forceinline__ DF s_from_f(float x) { return DF{x, 0.f}; }
__device__ __forceinline__ double s_val(double a) { return a; }
__device__ __forceinline__ double s_val(DF a) { return (double)a.hi + (double)a.lo; }
// to the vector precision (float pairs round to float without FP64 work)
__device__ __forceinline__ double s_to(double a) { return a; }
__device__ __forceinline__ float s_to(DF a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ double s_shfl_up(double v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ DF s_shfl_up(DF v, int d) {
    return DF{__shfl_up_sync(0xffffffffu, v.hi, d), __shfl_up_sync(0xffffffffu, v.lo, d)};
}
__device__ __forceinline__ double s_shfl(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ DF s_shfl(DF v, int l) {
    return DF{__shfl_sync(0xffffffffu, v.hi, l), __shfl_sync(0xffffffffu, v.lo, l)};
}
template <typename V>
__device__ __forceinline__ V s_zero() {
    return s_from<V>(0.0);
}
template <typename V, typename T>
__device__ __forceinline__ V s_of(T x);
template <>
__device__ __forceinline__ double s_of<double, double>(double x) { return x; }
template <>
__device__ __forceinline__ DF s_of<DF, float>(float x) { return DF{x, 0.f}; }

// Segmented sums: a pair (v, f) is a sum v that restarts at a head when f;
// combining a left pair with a right one gives (f_r ? v_r : v_l + v_r, f_l | f_r).
// Exclusive scan of one pair per thread over the block (fixed order): the
// carried pair into the thread (value and flag); *tv, *tf = the block's pair.
template <typename V>
__device__ inline V block_excl_seg_scan(V v, int f, int *cf, V *tv, int *tf) {
    __shared__ V wv[32];
    __shared__ int wf[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    V x = v;
    int g = f;
    for (int d = 1; d < 32; d <<= 1) {
        const V y = s_shfl_up(x, d);
        const int h = __shfl_up_sync(0xffffffffu, g, d);
        if (lane >= d) {
            if (!g) x = s_add(y, x);
            g |= h;
        }
    }
    V ex = s_shfl_up(x, 1);
    int exf = __shfl_up_sync(0xffffffffu, g, 1);
    if (lane == 0) {
        ex = s_zero<V>();
        exf = 0;
    }
    __syncthreads();
    if (lane == 31) {
        wv[wid] = x;
        wf[wid] = g;
    }
    __syncthreads();
    if (wid == 0) {
        V w = lane < nw ? wv[lane] : s_zero<V>();
        int wg = lane < nw ? wf[lane] : 0;
        for (int d = 1; d < 32; d <<= 1) {
            const V y = s_shfl_up(w, d);
            const int h = __shfl_up_sync(0xffffffffu, wg, d);
            if (lane >= d) {
                if (!wg) w = s_add(y, w);
                wg |= h;
            }
        }
        if (lane < nw) {
            wv[lane] = w;
            wf[lane] = wg;
        }
    }
    __syncthreads();
    V carry = wid > 0 ? wv[wid - 1] : s_zero<V>();
    const int carf = wid > 0 ? wf[wid - 1] : 0;
    if (exf) carry = ex;
    else carry = s_add(carry, ex);
    *cf = carf | exf;
    *tv = wv[nw - 1];
    *tf = wf[nw - 1];
    return carry;
}

// carry into every block b from blocks 0..b-1 (segmented), into shared memory
template <typename V>
__device__ inline void block_offsets_seg(const V *pv, const double *pf, V *off) {
    const int G = (int)gridDim.x;
    const int per = (G + (int)blockDim.x - 1) / (int)blockDim.x;
    const int i0 = (int)threadIdx.x * per;
    V v = s_zero<V>();
    int f = 0;
    for (int i = i0; i < i0 + per && i < G; ++i) {
        if (pf[i] != 0.0) {
            v = pv[i];
            f = 1;
        } else {
            v = s_add(v, pv[i]);
        }
    }
    int cf, tf;
    V tv;
    V run = block_excl_seg_scan(v, f, &cf, &tv, &tf);
    for (int i = i0; i < i0 + per && i < G; ++i) {
        off[i] = run;
        if (pf[i] != 0.0) run = pv[i];
        else run = s_add(run, pv[i]);
    }
    __syncthreads();
}

constexpr int kEuBatch = 8;   // consecutive tour positions per thread and tile

// One segmented scan pass over the block's stretch [b0, b1) of a sequence
// (the tour's positions, or the preorder's slots) with heads head[p]:
// S[p] = sum of val(p, head[p]) over [latest head <= p, p) inside the block
// (the carry from earlier blocks is added by the reader: it applies before
// the block's first head).  The stretch goes in tiles of blockDim * kEuBatch positions,
// kEuBatch consecutive ones per thread (coalesced; the values are gathered
// once and kept in registers); a segmented block scan per tile, the block's
// running pair carried from tile to tile.  Block pair into pv[b], pf[b];
// first head into fh[b].
template <typename T, typename VAL>
__device__ inline void euler_scan_pass(const uint8_t *head, int64_t b0, int64_t b1, VAL val,
                                       typename SumOf<T>::type *S, typename SumOf<T>::type *pv,
                                       double *pf, long long *fh) {
    using V = typename SumOf<T>::type;
    const int64_t tile = (int64_t)blockDim.x * kEuBatch;
    V cv = s_zero<V>();
    int cfl = 0;
    long long first = LLONG_MAX;
    for (int64_t base = b0; base < b1; base += tile) {
        const int64_t p0 = base + (int64_t)threadIdx.x * kEuBatch;
        uint8_t hd[kEuBatch];
        T x[kEuBatch];
#pragma unroll
        for (int k = 0; k < kEuBatch; ++k) hd[k] = p0 + k < b1 ? head[p0 + k] : 0;
#pragma unroll
        for (int k = 0; k < kEuBatch; ++k) x[k] = p0 + k < b1 ? val(p0 + k, hd[k] != 0) : (T)0;
        V sv = s_zero<V>();
        int sf = 0;
#pragma unroll
        for (int k = 0; k < kEuBatch; ++k) {
            if (hd[k]) {
                sv = s_zero<V>();
                sf = 1;
                if (first == LLONG_MAX) first = p0 + k;
            }
            sv = s_add(sv, s_of<V, T>(x[k]));
        }
        int carf, tf;
        V tvv;
        const V carry = block_excl_seg_scan(sv, sf, &carf, &tvv, &tf);
        V run = carf ? carry : s_add(cv, carry);
#pragma unroll
        for (int k = 0; k < kEuBatch; ++k) {
            if (p0 + k < b1) {
                if (hd[k]) run = s_zero<V>();
                S[p0 + k] = run;
                run = s_add(run, s_of<V, T>(x[k]));
            }
        }
        cv = tf ? tvv : s_add(cv, tvv);
        cfl |= tf;
    }
    // the block's first head: min over threads
    __shared__ long long s_first;
    __syncthreads();
    if (threadIdx.x == 0) s_first = LLONG_MAX;
    __syncthreads();
    if (first != LLONG_MAX) atomicMin(&s_first, first);
    __syncthreads();
    if (threadIdx.x == 0) {
        pv[blockIdx.x] = cv;
        pf[blockIdx.x] = cfl ? 1.0 : 0.0;
        fh[blockIdx.x] = s_first;
    }
}

// The preorder form (Y, the tour's per-vertex arrays and the heads in the
// tree's preorder; k's subtree is the slot range [k, k + size_k) with
// size_k = (out_k - in_k + 1) / 2):
//  1. S1 = exclusive prefix sums of b over the slots (0 at the roots),
//     restarting at every root;
//  2. c_k = (S1 inclusive at k + size_k - 1  -  S1 exclusive at k) / w_k;
//  3. d_k = c_k - sum of c_j over the vertices j whose subtrees end at
//     k - 1 (the tour's exits between the entries of k - 1 and k; none
//     after a root), 0 at the roots; S3 = exclusive prefix sums of d;
//  4. x_k = S3 at k + d_k: the sum of c over k's ancestors and k itself (the
//     slots j <= k whose subtree has not ended before k).
// Scans of n slots in place of 2 (n - roots) tour positions, read in order.
template <typename T>
__device__ __forceinline__ bool euler_solve_pre(const EulerKArgs &E, T *Y, unsigned int *bar,
                                             long long budget, int *err, unsigned int &epoch,
                                             double &mx, typename SumOf<T>::type *s_off) {
    using V = typename SumOf<T>::type;
    const int64_t G = gridDim.x, N = E.n;
    const int64_t per = (N + G - 1) / G;
    const int64_t b0 = min(N, (int64_t)blockIdx.x * per), b1 = min(N, b0 + per);
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    V *S = reinterpret_cast<V *>(E.S);
    T *C = reinterpret_cast<T *>(E.C);
    T *D = reinterpret_cast<T *>(E.D);
    V *pv = reinterpret_cast<V *>(E.part);
    double *pf = E.part + G;
    long long *fh = reinterpret_cast<long long *>(E.part + 2 * G);
    const T *ipw = reinterpret_cast<const T *>(E.ipw);
    const uint32_t per32 = (uint32_t)per;
    auto glob = [&](int64_t p, const long long *fhp) {
        const uint32_t b = (uint32_t)p / per32;
        return p < fhp[b] ? s_add(S[p], s_off[b]) : S[p];
    };
    const int64_t vbase = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // 1
    euler_scan_pass<T>(E.head_n, b0, b1, [&](int64_t p, bool hd) { return hd ? (T)0 : Y[p]; }, S,
                       pv, pf, fh);
    if (!grid_sync(bar, budget, err, epoch)) return false;
    // 2
    block_offsets_seg(pv, pf, s_off);
    for (int64_t v0 = vbase; v0 < N; v0 += nth * kEuBatch) {
        int32_t in[kEuBatch], out[kEuBatch];
#pragma unroll
        for (int k = 0; k < kEuBatch; ++k) {
            const int64_t v = v0 + k * nth;
            in[k] = v < N ? E.ein[v] : -1;
            out[k] = v < N ? E.eout[v] : -1;
        }
        T c[kEuBatch];
#pragma unroll
        for (int k = 0; k < kEuBatch; ++k) {
            const int64_t v = v0 + k * nth;
            c[k] = (T)0;
            if (in[k] >= 0) {
                const int64_t last = v + (out[k] - in[k] + 1) / 2 - 1;
                const V hi = s_add(glob(last, fh), s_of<V, T>(Y[last]));
                c[k] = (T)s_to(s_sub(hi, glob(v, fh))) * ipw[v];
            }
        }
#pragma unroll
        for (int k = 0; k < kEuBatch; ++k) {
            const int64_t v = v0 + k * nth;
            if (v < N) C[v] = c[k];
        }
    }
    if (!grid_sync(bar, budget, err, epoch)) return false;
    // 3
    euler_scan_pass<T>(E.head_n, b0, b1, [&](int64_t p, bool hd) {
        if (hd) {
            D[p] = (T)0;
            return (T)0;
        }
        T d = C[p];
        if (!E.head_n[p - 1]) {
            for (int32_t q = E.ein[p - 1] + 1; q < E.ein[p]; ++q) d -= C[-E.tour[q] - 1];
        }
        D[p] = d;
        return d;
    }, S, pv + 3 * G, pf + 3 * G, fh + 3 * G);
    if (!grid_sync(bar, budget, err, epoch)) return false;
    // 4, in the chunks of for_chunks: the one-column element loops that
    // follow read Y with this mapping, so no barrier is needed after it
    block_offsets_seg(pv + 3 * G, pf + 3 * G, s_off);
    T tm = (T)0;
    constexpr int W = Chunk<T>::W;
    for_chunks<T>(N, vbase, nth, [&](int64_t i0, int cnt) {
        T x[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const int64_t v = i0 + w;
            x[w] = w < cnt && !E.head_n[v] ? (T)s_to(s_add(glob(v, fh + 3 * G), s_of<V, T>(D[v])))
                                           : (T)0;
            tm = fmax(tm, fabs(x[w]));
        }
        st_chunk(Y + i0, cnt, x);
    });
    mx = fmax(mx, (double)tm);
    return true;
}

template <typename T>
__device__ __forceinline__ bool euler_solve_tour(const EulerKArgs &E, T *Y, unsigned int *bar,
                                                long long budget, int *err, unsigned int &epoch,
                                                double &mx, typename SumOf<T>::type *s_off) {
    using V = typename SumOf<T>::type;
    const int64_t G = gridDim.x;
    const int64_t per = (E.L + G - 1) / G;
    const int64_t b0 = min(E.L, (int64_t)blockIdx.x * per), b1 = min(E.L, b0 + per);
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    V *S = reinterpret_cast<V *>(E.S);
    T *C = reinterpret_cast<T *>(E.C);
    V *pv = reinterpret_cast<V *>(E.part);
    double *pf = E.part + G;
    long long *fh = reinterpret_cast<long long *>(E.part + 2 * G);
    const T *ipw = reinterpret_cast<const T *>(E.ipw);
    // global prefix at p: the block-local part, plus the carry from earlier
    // blocks while p lies before the block's first head (block of a position:
    // 32-bit division, positions < 2^31)
    const uint32_t per32 = (uint32_t)per;
    auto glob = [&](int64_t p, const long long *fhp) {
        const uint32_t b = (uint32_t)p / per32;
        return p < fhp[b] ? s_add(S[p], s_off[b]) : S[p];
    };
    const int64_t vbase = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // 1: prefix sums of b at the entries, restarting at every tree
    euler_scan_pass<T>(E.head, b0, b1, [&](int64_t p, bool) {
        const int32_t v = E.tour[p];
        return v >= 0 ? Y[v] : (T)0;
    }, S, pv, pf, fh);
    if (!grid_sync(bar, budget, err, epoch)) return false;
    // 2: currents c_v = (subtree sum of b) / w_v
    block_offsets_seg(pv, pf, s_off);
    for (int64_t v0 = vbase; v0 < E.n; v0 += nth * kEuBatch) {
        int32_t in[kEuBatch], out[kEuBatch];
#pragma unroll
        for (int k = 0; k < kEuBatch; ++k) {
            const int64_t v = v0 + k * nth;
            in[k] = v < E.n ? E.ein[v] : -1;
            out[k] = v < E.n ? E.eout[v] : -1;
        }
        T d[kEuBatch];
#pragma unroll
        for (int k = 0; k < kEuBatch; ++k)
            d[k] = in[k] >= 0 ? (T)s_to(s_sub(glob(out[k], fh), glob(in[k], fh))) : (T)0;
#pragma unroll
        for (int k = 0; k < kEuBatch; ++k) {
            const int64_t v = v0 + k * nth;
            if (v < E.n) C[v] = in[k] >= 0 ? d[k] * ipw[v] : (T)0;
        }
    }
    if (!grid_sync(bar, budget, err, epoch)) return false;
    // 3: prefix sums of +c at entries, -c at exits, restarting at every tree
    euler_scan_pass<T>(E.head, b0, b1, [&](int64_t p, bool) {
        const int32_t v = E.tour[p];
        return v >= 0 ? C[v] : -C[-v - 1];
    }, S, pv + 3 * G, pf + 3 * G, fh + 3 * G);
    if (!grid_sync(bar, budget, err, epoch)) return false;
    // 4: x_v = the path sum up to and including v's entry (roots: 0)
    block_offsets_seg(pv + 3 * G, pf + 3 * G, s_off);
    T tm = (T)0;
    for (int64_t v0 = vbase; v0 < E.n; v0 += nth * kEuBatch) {
        int32_t in[kEuBatch];
#pragma unroll
        for (int k = 0; k < kEuBatch; ++k) {
            const int64_t v = v0 + k * nth;
            in[k] = v < E.n ? E.ein[v] : -1;
        }
        T x[kEuBatch];
#pragma unroll
        for (int k = 0; k < kEuBatch; ++k) {
            const int64_t v = v0 + k * nth;
            x[k] = in[k] >= 0 ? (T)s_to(s_add(glob(in[k], fh + 3 * G), s_of<V, T>(C[v]))) : (T)0;
        }
#pragma unroll
        for (int k = 0; k < kEuBatch; ++k) {
            const int64_t v = v0 + k * nth;
            if (v >= E.n) continue;
            Y[v] = x[k];
            tm = fmax(tm, fabs(x[k]));
        }
    }
    mx = fmax(mx, (double)tm);
    return true;
}


// PRE: the preorder form (E.pre set by euler_kargs), else the tour form.
template <typename T, bool PRE = false>
__device__ __forceinline__ bool euler_solve_dev(const EulerKArgs &E, T *Y, unsigned int *bar,
                                                long long budget, int *err, unsigned int &epoch,
                                                double &mx) {
    __shared__ typename SumOf<T>::type s_off[kEulerMaxGrid];
    if constexpr (PRE) return euler_solve_pre<T>(E, Y, bar, budget, err, epoch, mx, s_off);
    else return euler_solve_tour<T>(E, Y, bar, budget, err, epoch, mx, s_off);
}

// Host side: scan-form arguments for a cooperative grid of `grid` blocks;
// pre: the vectors are in the tree's preorder numbering (else vertex ids).
template <typename T>
inline void euler_kargs(grass_ctx_t ctx, const grass_tree_s *Tr, int grid, EulerKArgs *e,
                        bool pre = false) {
    if (grid > kEulerMaxGrid) fail(GRASS_ERR_INVALID, "grid too large for the scan-form tree solve");
    const EulerTour &E = Tr->euler;
    e->L = E.L;
    e->n = Tr->g.n;
    e->tour = pre ? E.tour_pre.p : E.tour.p;
    e->ein = pre ? E.ein_pre.p : E.ein.p;
    e->eout = pre ? E.eout_pre.p : E.eout.p;
    e->head = E.head.p;
    e->pre = pre ? 1 : 0;
    e->head_n = pre ? E.head_pre.p : nullptr;
    e->D = pre ? (void *)ctx->scr<double>(SCR_EU_A, Tr->g.n) : nullptr;
    if constexpr (sizeof(T) == 8) e->ipw = pre ? E.ipw_pre.p : E.ipw.p;
    else e->ipw = pre ? E.ipw32_pre.p : E.ipw32.p;
    e->S = ctx->scr<double>(SCR_EU_S, E.L + 1);   // 8-byte sums (double or float pair)
    e->C = ctx->scr<double>(SCR_EU_C, Tr->g.n);
    e->part = ctx->scr<double>(SCR_EU_P, 6 * (size_t)grid + 2);
}

// Grid of a cooperative kernel with `threads` threads and `smem` dynamic
// shared memory: co-resident blocks per SM, capped by tree_blocks_per_sm, and
// no more blocks than `work_threads` threads of work fill (small graphs leave
// the other SMs free and their grid barriers have fewer arrivals), on at
// most grid_sms SMs when that knob is set.  The grid is a function of the
// shape, the work and the knobs only, so a result does not depend on what
// else runs on the device.
template <typename K>
inline int coop_grid(grass_ctx_t ctx, K kernel, int threads, size_t smem, int64_t work_threads) {
    const void *k = (const void *)kernel;
    int per_sm = 0;
    for (const auto &e : ctx->coop_cache)
        if (e.kernel == k && e.threads == threads && e.smem == smem && e.bpsm == ctx->tree_bpsm)
            per_sm = e.grid;
    if (per_sm == 0) {
        GCK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmem));
        int nb = 0;
        GCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem));
        if (nb < 1) fail(GRASS_ERR_CUDA, "cooperative kernel does not fit on an SM");
        per_sm = std::min(nb, ctx->tree_bpsm);
        ctx->coop_cache.push_back({k, threads, smem, ctx->tree_bpsm, per_sm});
    }
    // grid_sms: a share of the device (requests served side by side)
    const int sms = ctx->grid_sms > 0 ? std::min(ctx->grid_sms, ctx->num_sms) : ctx->num_sms;
    const int64_t full = (int64_t)sms * per_sm;
    const int64_t need = std::max<int64_t>(1, (work_threads + threads - 1) / threads);
    return (int)std::min<int64_t>(full, need);
}

// Host side: the arguments of one solve on tree T with factor f, and the
// dynamic shared memory its tail needs.
template <typename T, int R>
inline TreeKArgs<T> tree_kargs(grass_ctx_t ctx, const grass_tree_s *Tr, const TreeFactor &f,
                               size_t *smem) {
    const TreeSchedule &S = Tr->sched;
    auto alive_at = [&](int k) { return S.tail_n - (S.elim_off[k] - S.elim_off[S.tail_k0]); };
    // the tail's rows and its records / coefficients must fit the budget,
    // and its work (vertices x max(1, r/4)) stay within tree_tail_items
    auto tail_bytes = [&](int k) {
        return TailSmem<T, R>::bytes(alive_at(k), S.rcv_off[S.rounds] - S.rcv_off[k],
                                     S.elim_off[S.rounds] - S.elim_off[k],
                                     S.contrib_off[S.rounds] - S.contrib_off[k]);
    };
    int K1 = S.tail_k0;
    while (K1 < S.rounds && (tail_bytes(K1) > kTailSmem ||
                             alive_at(K1) * std::max(1, R / 4) > std::max<int64_t>(ctx->tree_tail_items, 1)))
        ++K1;
    const int64_t ntl = alive_at(K1);
    *smem = tail_bytes(K1);
    TreeKArgs<T> ka;
    ka.rounds = S.rounds;
    ka.K1 = K1;
    ka.base = S.tail_n - ntl;
    ka.ntl = ntl;
    ka.r0 = S.rcv_off[S.tail_k0];
    ka.e0 = S.elim_off[S.tail_k0];
    ka.c0 = S.tail_c0;
    ka.tf0 = S.rcv_off[K1];
    ka.tnf = S.rcv_off[S.rounds] - S.rcv_off[K1];
    ka.tg0 = S.elim_off[K1];
    ka.tnb = S.elim_off[S.rounds] - S.elim_off[K1];
    ka.tc0 = S.contrib_off[K1];
    ka.ntc = S.contrib_off[S.rounds] - S.contrib_off[K1];
    ka.rcv_off = S.d_offs.p;
    ka.elim_off = S.d_offs.p + (S.rounds + 1);
    ka.fwd_rec = S.fwd_rec.p;
    ka.bwd_rec = S.bwd_rec.p;
    ka.fwd_loc = S.fwd_loc.p;
    ka.bwd_loc = S.bwd_loc.p;
    if constexpr (sizeof(T) == 8) {
        ka.fm = f.fm64.p;
        ka.bc = f.bc64.p;
        ka.cm = f.cm64.p;
    } else {
        ka.fm = f.fm32.p;
        ka.bc = f.bc32.p;
        ka.cm = f.cm32.p;
    }
    ka.beg = S.rcv_beg.p;
    ka.cv = S.contrib_v.p;
    ka.tail_vid = S.tail_vid.p;
    ka.contrib_loc = S.contrib_loc.p;
    if constexpr (sizeof(T) == 8) ka.root_invd = f.rinv64.p;
    else ka.root_invd = f.rinv32.p;
    ka.nroots = (int)Tr->nroots;
    ka.bar = ctx->gbar.p;
    ka.budget = ctx->wait_budget;
    ka.err = ctx->flags.p + 3;
    return ka;
}

}  // namespace grass
