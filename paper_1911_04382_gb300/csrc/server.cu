// server.cu -- the serving form: a request loop that admits sparsify-and-solve
// requests of uneven sizes by device-memory footprint and runs several at
// once on one GPU (continuous batching).
//
// Each worker ("slot") owns a context on its own non-blocking stream.  A
// request is admitted when a slot is idle and its footprint fits in what
// the budget has left; requests are taken in arrival order (the oldest
// waiting request goes first; while it does not fit, the ones behind it
// wait too, so large requests are not starved).  An admitted request keeps
// its inputs, tree, sparsifier and Krylov state on the device until it
// completes; its kernels run on the slot's stream, so the work of the
// requests in flight overlaps on the device.  Every launch shape depends on
// the request alone, never on what else runs, so a result is the same alone
// and in the mix.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace grass {
namespace {

using Clock = std::chrono::steady_clock;

struct Ticket {
    int64_t id = 0;
    grass_request_t req{};
    grass_result_t res{};
    int64_t footprint = 0;
    bool done = false;
};

struct DevMem {
    void *p = nullptr;
    ~DevMem() {
        if (p) cudaFree(p);
    }
    void *alloc(size_t bytes) {
        GCK(cudaMalloc(&p, bytes ? bytes : 1));
        return p;
    }
};

void set_error(grass_result_t &r, grass_status st, const char *msg) {
    r.status = st;
    snprintf(r.error, sizeof(r.error), "%s", msg ? msg : "");
}

}  // namespace
}  // namespace grass

struct grass_server_s {
    int device = 0;
    int64_t budget = 0, in_use = 0;
    std::mutex mu;
    std::condition_variable cv_admit, cv_done;
    std::deque<std::shared_ptr<grass::Ticket>> queue;
    std::unordered_map<int64_t, std::shared_ptr<grass::Ticket>> tickets;
    std::vector<std::thread> workers;
    bool stop = false;
    int64_t next_id = 1;
    int64_t running = 0, max_running = 0;
    std::atomic<int> grid_sms{0};   // cooperative grids of every request (0: all SMs)
    grass::Clock::time_point t0;

    double now() const {
        return std::chrono::duration<double>(grass::Clock::now() - t0).count();
    }
    void worker(int slot);
    void run(int slot, grass_ctx_t ctx, grass::Ticket &t);
};

using namespace grass;

// Bytes the device holds for one request: its inputs and outputs (CSR,
// h0, v0, b, x) plus what the library allocates for the tree, the
// sparsifier, the embedding blocks and the Krylov vectors.  The per-vertex,
// per-nonzero and per-column terms are upper bounds of the library's
// allocations (checked against measured use by the tests).
extern "C" int64_t grass_server_footprint(int64_t n, int64_t nnz, int r, int rounds) {
    if (n <= 0 || nnz < 0 || r <= 0 || rounds <= 0) return -1;
    const int64_t inputs = 8 * (n + 1) + 12 * nnz + 8 * n * r * (int64_t)rounds +
                           8 * n * (int64_t)rounds + 16 * n;
    const int64_t library = 600 * n + 40 * nnz + 48 * n * (int64_t)r;
    return inputs + library + (64LL << 20);
}

void grass_server_s::run(int slot, grass_ctx_t ctx, Ticket &t) {
    const grass_request_t &q = t.req;
    grass_result_t &res = t.res;
    GCK(cudaSetDevice(device));
    cudaStream_t s = ctx->stream;
    const int64_t n = q.n, nnz = q.nnz;
    const int rounds = q.params.max_rounds, r = q.params.r;
    DevMem rp, col, val, h0, v0, b, x;
    rp.alloc(8 * (n + 1));
    col.alloc(4 * nnz);
    val.alloc(8 * nnz);
    h0.alloc(8 * n * r * (int64_t)rounds);
    v0.alloc(8 * n * (int64_t)rounds);
    b.alloc(8 * n);
    x.alloc(8 * n);
    GCK(cudaMemcpyAsync(rp.p, q.rowptr, 8 * (n + 1), cudaMemcpyHostToDevice, s));
    GCK(cudaMemcpyAsync(col.p, q.col, 4 * nnz, cudaMemcpyHostToDevice, s));
    GCK(cudaMemcpyAsync(val.p, q.val, 8 * nnz, cudaMemcpyHostToDevice, s));
    GCK(cudaMemcpyAsync(h0.p, q.h0, 8 * n * r * (int64_t)rounds, cudaMemcpyHostToDevice, s));
    GCK(cudaMemcpyAsync(v0.p, q.v0, 8 * n * (int64_t)rounds, cudaMemcpyHostToDevice, s));
    GCK(cudaMemcpyAsync(b.p, q.b, 8 * n, cudaMemcpyHostToDevice, s));
    GCK(cudaStreamSynchronize(s));
    const double t_in = now();
    grass_csr_t A{n, nnz, (const int64_t *)rp.p, (const int32_t *)col.p, (const double *)val.p};
    grass_tree_t tree = nullptr;
    grass_sparsifier_t S = nullptr;
    grass_status st = grass_build_tree(ctx, &A, 0, &tree);
    const double t_tree = now();
    if (st == GRASS_OK) st = grass_densify(ctx, tree, &q.params, (const double *)h0.p,
                                           (const double *)v0.p, &S, &res.sparsify);
    const double t_dens = now();
    if (st == GRASS_OK) {
        st = grass_pcg_solve(ctx, S, (const double *)b.p, (double *)x.p, q.tol, q.maxit,
                             q.pcg_prec, q.refine_tol, q.pcg_inner_tol, q.pcg_inner_maxit,
                             &res.solve);
        if (st == GRASS_OK || st == GRASS_ERR_NOT_CONVERGED) {
            GCK(cudaMemcpyAsync(q.x, x.p, 8 * n, cudaMemcpyDeviceToHost, s));
            GCK(cudaStreamSynchronize(s));
        }
    }
    const double t_pcg = now();
    set_error(res, st, st == GRASS_OK ? "" : grass_last_error(ctx));
    if (S) grass_sparsifier_destroy(S);
    if (tree) grass_tree_destroy(tree);
    // scratch grows with the largest request a context has served: give it
    // back so the budget accounts for this request alone
    for (auto &sc : ctx->scratch) sc.release();
    res.ms_h2d = 1e3 * (t_in - res.t_admit);
    res.ms_tree = 1e3 * (t_tree - t_in);
    res.ms_densify = 1e3 * (t_dens - t_tree);
    res.ms_pcg = 1e3 * (t_pcg - t_dens);
    res.slot = slot;
}

void grass_server_s::worker(int slot) {
    grass_ctx_t ctx = nullptr;
    cudaStream_t s = nullptr;
    bool ok = cudaSetDevice(device) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
              grass_ctx_create(&ctx, s) == GRASS_OK;
    for (;;) {
        std::shared_ptr<Ticket> t;
        {
            std::unique_lock<std::mutex> lock(mu);
            cv_admit.wait(lock, [&] {
                return stop || (!queue.empty() && in_use + queue.front()->footprint <= budget);
            });
            if (queue.empty() || (stop && queue.empty())) break;
            if (stop && in_use + queue.front()->footprint > budget) break;
            t = queue.front();
            queue.pop_front();
            in_use += t->footprint;
            t->res.t_admit = now();
            running += 1;
            max_running = std::max(max_running, running);
            t->res.in_flight_at_admit = (int)running;
        }
        // the next request in line may fit beside this one
        cv_admit.notify_all();
        if (!ok) {
            set_error(t->res, GRASS_ERR_CUDA, "worker could not create its context");
        } else {
            try {
                if (grass_ctx_set_param(ctx, "grid_sms", grid_sms.load()) != GRASS_OK)
                    fail(GRASS_ERR_INVALID, "grid_sms rejected");
                run(slot, ctx, *t);
            } catch (const Error &e) {
                set_error(t->res, e.st, e.msg.c_str());
                for (auto &sc : ctx->scratch) sc.release();
            } catch (...) {
                set_error(t->res, GRASS_ERR_CUDA, "unexpected internal error");
            }
        }
        {
            std::lock_guard<std::mutex> lock(mu);
            in_use -= t->footprint;
            running -= 1;
            t->res.t_done = now();
            t->done = true;
        }
        cv_done.notify_all();
        cv_admit.notify_all();
    }
    if (ctx) grass_ctx_destroy(ctx);
    if (s) cudaStreamDestroy(s);
}

extern "C" grass_status grass_server_set_param(grass_server_t srv, const char *name, int64_t value) {
    if (!srv || !name) return GRASS_ERR_INVALID;
    if (std::string(name) == "grid_sms") {
        if (value < 0 || value > (1 << 20)) return GRASS_ERR_INVALID;
        srv->grid_sms.store((int)value);
        return GRASS_OK;
    }
    return GRASS_ERR_INVALID;
}

extern "C" grass_status grass_server_create(int device, int slots, int64_t hbm_budget,
                                            grass_server_t *out) {
    if (!out || slots < 1 || slots > 64) return GRASS_ERR_INVALID;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return GRASS_ERR_INVALID;
    }
    if (cudaSetDevice(device) != cudaSuccess) return GRASS_ERR_CUDA;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return GRASS_ERR_CUDA;
    auto *srv = new (std::nothrow) grass_server_s();
    if (!srv) return GRASS_ERR_OOM;
    srv->device = device;
    srv->budget = hbm_budget > 0 ? std::min<int64_t>(hbm_budget, (int64_t)free_b)
                                 : (int64_t)(0.85 * (double)free_b);
    srv->t0 = Clock::now();
    try {
        for (int i = 0; i < slots; ++i) srv->workers.emplace_back(&grass_server_s::worker, srv, i);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lock(srv->mu);
            srv->stop = true;
        }
        srv->cv_admit.notify_all();
        for (auto &w : srv->workers) w.join();
        delete srv;
        return GRASS_ERR_CUDA;
    }
    *out = srv;
    return GRASS_OK;
}

extern "C" int64_t grass_server_budget(grass_server_t srv) { return srv ? srv->budget : -1; }

extern "C" grass_status grass_server_submit(grass_server_t srv, const grass_request_t *req,
                                            int64_t *ticket) {
    if (!srv || !req || !ticket) return GRASS_ERR_INVALID;
    const grass_request_t &q = *req;
    if (q.n < 2 || q.nnz < q.n || !q.rowptr || !q.col || !q.val || !q.h0 || !q.v0 || !q.b || !q.x ||
        q.params.r < 1 || q.params.r > 32 || q.params.max_rounds < 1 ||
        q.params.max_rounds > GRASS_MAX_ROUNDS)
        return GRASS_ERR_INVALID;
    auto t = std::make_shared<Ticket>();
    t->req = q;
    t->footprint = grass_server_footprint(q.n, q.nnz, q.params.r, q.params.max_rounds);
    std::lock_guard<std::mutex> lock(srv->mu);
    if (srv->stop) return GRASS_ERR_INVALID;
    if (t->footprint > srv->budget) return GRASS_ERR_OOM;   // would never be admitted
    t->id = srv->next_id++;
    t->res.footprint_bytes = t->footprint;
    t->res.t_submit = srv->now();
    srv->tickets[t->id] = t;
    srv->queue.push_back(t);
    *ticket = t->id;
    srv->cv_admit.notify_all();
    return GRASS_OK;
}

extern "C" grass_status grass_server_wait(grass_server_t srv, int64_t ticket, grass_result_t *out) {
    if (!srv || !out) return GRASS_ERR_INVALID;
    std::unique_lock<std::mutex> lock(srv->mu);
    auto it = srv->tickets.find(ticket);
    if (it == srv->tickets.end()) return GRASS_ERR_INVALID;
    std::shared_ptr<Ticket> t = it->second;
    srv->cv_done.wait(lock, [&] { return t->done; });
    *out = t->res;
    srv->tickets.erase(ticket);
    return GRASS_OK;
}

extern "C" grass_status grass_server_stats(grass_server_t srv, int64_t *in_use, int64_t *queued,
                                           int64_t *running, int64_t *max_running) {
    if (!srv) return GRASS_ERR_INVALID;
    std::lock_guard<std::mutex> lock(srv->mu);
    if (in_use) *in_use = srv->in_use;
    if (queued) *queued = (int64_t)srv->queue.size();
    if (running) *running = srv->running;
    if (max_running) *max_running = srv->max_running;
    return GRASS_OK;
}

extern "C" void grass_server_destroy(grass_server_t srv) {
    if (!srv) return;
    {
        std::unique_lock<std::mutex> lock(srv->mu);
        srv->cv_done.wait(lock, [&] { return srv->queue.empty() && srv->running == 0; });
        srv->stop = true;
    }
    srv->cv_admit.notify_all();
    for (auto &w : srv->workers) w.join();
    delete srv;
}
