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
#include <cuda.h>

#include <mutex>
#include <utility>
#include <vector>

#include "tree_solve.cuh"

namespace grass {
namespace {

// [0] barrier arrival counter, [2] barrier hold flag (the context's
// setting, copied in by every call), [8] wait-timeout flag; the rest is
// unused.  One array per device, shared by every call on that device.
constexpr int kNoallocWords = 64;
static __device__ __align__(256) unsigned int g_noalloc_scratch[kNoallocWords];

// The array's device address, looked up once per CUDA context (that is, per
// device, and again if the application resets the device and the module is
// loaded into a new context).  Contexts are told apart by their driver id,
// which is never reused within a process; the two driver calls are taken
// through the runtime's entry-point query, so the library needs no link
// against the driver library.
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

std::mutex g_addr_mu;
std::vector<std::pair<unsigned long long, unsigned int *>> g_addr;   // (context id, address)
CtxGetCurrentFn g_get_current = nullptr;
CtxGetIdFn g_get_id = nullptr;

unsigned long long current_context_id() {
    if (!g_get_current || !g_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        GCK(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1));
        GCK(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2));
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            fail(GRASS_ERR_CUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId not found");
        g_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        g_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (g_get_current(&c) != CUDA_SUCCESS || !c || g_get_id(c, &id) != CUDA_SUCCESS)
        fail(GRASS_ERR_CUDA, "no current CUDA context");
    return id;
}

// Device address of the array in the current context (the caller has made
// the context's device current).
unsigned int *scratch_address() {
    std::lock_guard<std::mutex> lock(g_addr_mu);
    const unsigned long long id = current_context_id();
    for (const auto &e : g_addr)
        if (e.first == id) return e.second;
    void *p = nullptr;
    GCK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_addr.emplace_back(id, static_cast<unsigned int *>(p));
    return g_addr.back().second;
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
        unsigned int *scratch = scratch_address();
        const size_t bytes = (size_t)T->g.n * r * (prec == GRASS_FP64 ? 8 : 4);
        if (B != X)
            GCK(cudaMemcpyAsync(X, B, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        // the array keeps the previous call's counter and flag: start both at
        // zero; the hold flag follows grass_ctx_set_wait_limit on ctx
        GCK(cudaMemsetAsync(scratch, 0, kNoallocWords * sizeof(unsigned int), ctx->stream));
        GCK(cudaMemcpyAsync(scratch + 2, ctx->gbar.p + 2, sizeof(unsigned int),
                            cudaMemcpyDeviceToDevice, ctx->stream));
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
