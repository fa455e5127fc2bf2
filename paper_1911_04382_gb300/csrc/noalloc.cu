// noalloc.cu -- a tree solve that allocates no device memory.
//
// grass_tree_solve takes its grid-barrier counter and its wait-timeout flag
// from buffers the context allocated.  Some callers cannot have the library
// allocate once they run: code with a fixed device-memory budget that has
// already handed the rest of the GPU to another allocator (a framework's
// caching pool that must see every byte), and latency-bound loops that may
// not call cudaMalloc or cudaFree at all, because those calls synchronise the
// device.  grass_tree_solve_noalloc gives them the same solve with its
// scratch in the file-scope array below: 256 bytes that every GPU which loads
// this library holds until the process exits, whatever the tree's size.
#include <mutex>

#include "tree_solve.cuh"

namespace grass {
namespace {

// [0] barrier arrival counter, [2] barrier hold flag (always 0 here),
// [8] wait-timeout flag; the rest is unused.  One array per device, shared
// by every call on that device.
constexpr int kNoallocWords = 64;
static __device__ __align__(256) unsigned int g_noalloc_scratch[kNoallocWords];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
unsigned int *g_addr[kMaxDevices] = {nullptr};

// Device address of the array on device `dev`, looked up on the first call
// there (that device must be current).
unsigned int *scratch_address(int dev) {
    if (dev < 0 || dev >= kMaxDevices) fail(GRASS_ERR_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        GCK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_addr[dev] = static_cast<unsigned int *>(p);
    }
    return g_addr[dev];
}

template <typename T, int R>
__global__ void __launch_bounds__(kPersistMaxThreads, 1)
    k_tree_noalloc(TreeKArgs<T> a, T *Y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned int epoch = 0;
    double mx = 0.0;
    tree_tail_stage<T, R>(a, reinterpret_cast<T *>(smem_raw));
    tree_solve_dev<T, R>(a, Y, epoch, mx, reinterpret_cast<T *>(smem_raw));
}

struct NoallocCall {
    grass_ctx_t ctx;
    grass_tree_t T;
    const TreeFactor *f;
    void *Y;
    grass_prec prec;
    unsigned int *scratch;
};

// Every call zeroes the counter, and each grid barrier adds one arrival per
// block to it: the count must stay inside 32 bits.
constexpr int64_t kMaxArrivals = int64_t(1) << 31;

template <typename T, int R>
void launch_noalloc(const NoallocCall &c) {
    grass_ctx_t ctx = c.ctx;
    size_t smem = 0;
    TreeKArgs<T> ka = tree_kargs<T, R>(ctx, c.T, *c.f, &smem);
    ka.bar = c.scratch;
    ka.err = reinterpret_cast<int *>(c.scratch + 8);
    const int grid = coop_grid(ctx, k_tree_noalloc<T, R>, ctx->tree_threads, smem,
                               c.T->g.n * Lay<R>::TPR);
    if ((int64_t)grid * (2 * (int64_t)ka.rounds + 2) >= kMaxArrivals)
        fail(GRASS_ERR_INVALID, "tree schedule too long for the no-allocation barrier counter");
    T *Y = static_cast<T *>(c.Y);
    void *args[] = {&ka, &Y};
    GCK(cudaLaunchCooperativeKernel((const void *)k_tree_noalloc<T, R>, dim3(grid),
                                    dim3(ctx->tree_threads), args, smem, ctx->stream));
    ctx->launches++;
}

template <int R>
void noalloc_R(const NoallocCall &c) {
    if (c.prec == GRASS_FP64) launch_noalloc<double, R>(c);
    else launch_noalloc<float, R>(c);
}

void reject(bool ok, const char *msg) {
    if (!ok) fail(GRASS_ERR_INVALID, msg);
}

}  // namespace
}  // namespace grass

using namespace grass;

extern "C" grass_status grass_tree_solve_noalloc(grass_ctx_t ctx, grass_tree_t T, int with_D,
                                                  int r, grass_prec prec, const void *B, void *X) {
    if (!ctx || !T) return GRASS_ERR_INVALID;
    try {
        GCK(cudaSetDevice(ctx->device));
        reject(B && X, "null block");
        reject(prec == GRASS_FP64 || prec == GRASS_FP32, "prec must be GRASS_FP64 or GRASS_FP32");
        reject(r_supported(r), "r must be 1, 2, 4, 8, 16, 24 or 32");
        reject(ctx->num_sms > 0, "the device cannot launch cooperative kernels");
        reject(!with_D || T->has_sdd,
               "the L_T + D factor is not built; one grass_tree_solve call with with_D=1 builds it");
        unsigned int *scratch = scratch_address(ctx->device);
        const size_t bytes = (size_t)T->g.n * r * (prec == GRASS_FP64 ? 8 : 4);
        if (B != X)
            GCK(cudaMemcpyAsync(X, B, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        // the array keeps the previous call's counter and flag: start both at zero
        GCK(cudaMemsetAsync(scratch, 0, kNoallocWords * sizeof(unsigned int), ctx->stream));
        NoallocCall c{ctx, T, with_D ? &T->sdd : &T->lap, X, prec, scratch};
        GRASS_DISPATCH_R(r, noalloc_R, c);
        int timed_out = 0;
        GCK(cudaMemcpyAsync(&timed_out, scratch + 8, sizeof(int), cudaMemcpyDeviceToHost,
                            ctx->stream));
        GCK(cudaStreamSynchronize(ctx->stream));
        if (timed_out) fail(GRASS_ERR_TIMEOUT, "a bounded device-side wait expired (grid barrier)");
    } catch (const Error &e) {
        ctx->err = e.msg;
        return e.st;
    } catch (...) {
        ctx->err = "unexpected internal error";
        return GRASS_ERR_CUDA;
    }
    return GRASS_OK;
}
