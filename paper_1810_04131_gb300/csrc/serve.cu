// Serving: independent particle configurations submitted as requests and
// solved (label, Eq. bie, forces and torques) by the library with
// continuous batching.
//
// A worker that admits a small mixed-precision request (up to
// SMALL_REQUEST_NODES nodes, dense far field, block preconditioner) also
// admits the small ones queued right behind it, up to MAX_BATCH, and solves
// them together: their inner FP32 GMRES advance in lock step, one kernel
// launch per stage for all of them (batch.cu). Larger requests run alone.
//
// A fixed set of worker slots, each with its own CUDA streams (a
// high-priority one for small requests, a low-priority one for large ones)
// and internal context, takes requests from the arrival queue. A request is admitted when
// a slot is free and its device-memory estimate fits the budget left by the
// requests in flight; requests that arrive while others run are admitted as
// soon as a slot and memory free up, and their kernels overlap on the
// device (one stream per slot). Results are copied to host memory and kept
// until yk_poll collects them. Host waits are bounded: yk_drain gives up
// when no request has completed for five minutes and reports YK_ERR_TIMEOUT.
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "yk_internal.cuh"

namespace yk {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    std::vector<yk_particle> parts;
    yk_params prm{};
    int label_kind = YK_LABEL_TANH;
    double label_param = 10.0;
    int status = YK_REQ_QUEUED;
    int error = YK_OK;
    size_t mem_bytes = 0;
    Clock::time_point t_submit, t_done;
    std::vector<double> sigma, F, tau;
    yk_solve_info info{};
};

struct Server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    uint64_t next_id = 1;
    std::deque<uint64_t> queue;                       // arrival order
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    size_t max_queue = 1 << 16;
    size_t mem_budget = 0, mem_in_flight = 0;
    int running = 0;
    uint64_t finished = 0;                           // requests completed so far
    bool stop = false;
    std::vector<std::thread> workers;
    int device = 0;
};

// Device memory of one request: node arrays, Krylov basis (and its
// preconditioned copy), chunk partials,
// scratch vectors, QBX rows, per shape (at most two) the two self blocks and
// the FP64 + FP32 preconditioner inverse and the inner GMRES's coarse space
// (an estimate with a safety factor).
static size_t request_bytes(const Request& r) {
    const size_t npp = (size_t)r.prm.n_panels * r.prm.n_gl;
    const size_t n = (size_t)r.parts.size() * npp;
    const size_t m = (size_t)r.prm.gmres_restart;
    const size_t nchunk = 32;
    const size_t rows = npp * 9 * r.prm.n_gl * 2;
    const size_t blocks = 2 * npp * npp * (8 * 2 + 8 + 4);
    const size_t coarse = coarse_bytes(r.parts.data(), (int)r.parts.size(), r.prm);
    return (size_t)(1.25 * (8.0 * (double)(n * (2 * m + 1 + nchunk + 16) + rows) + (double)blocks +
                            (double)coarse)) +
           (8u << 20);
}

// Requests up to this many nodes run on a high-priority stream, so that
// their blocks are scheduled ahead of those of large requests sharing the GPU,
// and, when they are mixed-precision dense-far-field solves, are batched.
constexpr int64_t SMALL_REQUEST_NODES = 65536;
constexpr int MAX_BATCH = 16;   // requests solved together by one worker

static int64_t request_nodes(const Request* r) {
    return (int64_t)r->parts.size() * r->prm.n_panels * r->prm.n_gl;
}

static bool batchable(const Request* r) {
    return request_nodes(r) <= SMALL_REQUEST_NODES && r->prm.precision == YK_MIXED &&
           r->prm.farfield == YK_FARFIELD_DENSE && r->prm.precond == YK_PRECOND_BLOCK;
}

// Run several requests together: geometries and data per request, one
// batched solve (lock-step inner GMRES, see batch.cu), forces per request.
// Returns per request its code in rc[].
static void run_batch(yk_ctx* ctx, const std::vector<Request*>& rs, std::vector<int>& rc) {
    const size_t k = rs.size();
    rc.assign(k, YK_OK);
    std::vector<yk_geom*> g(k, nullptr);
    std::vector<double*> f(k, nullptr), sig(k, nullptr), F(k, nullptr), tau(k, nullptr);
    cudaStream_t st = ctx->stream;
    std::vector<yk_geom*> ok_g;
    std::vector<const double*> ok_f;
    std::vector<double*> ok_s;
    std::vector<size_t> ok_i;
    for (size_t q = 0; q < k; ++q) {
        Request* r = rs[q];
        int c = yk_create_geometry(ctx, r->parts.data(), (int)r->parts.size(), &r->prm, &g[q]);
        if (c == YK_OK) {
            const size_t n = (size_t)g[q]->n, np = (size_t)g[q]->np;
            if (cudaMallocAsync((void**)&f[q], n * sizeof(double), st) != cudaSuccess ||
                cudaMallocAsync((void**)&sig[q], n * sizeof(double), st) != cudaSuccess ||
                cudaMallocAsync((void**)&F[q], 2 * np * sizeof(double), st) != cudaSuccess ||
                cudaMallocAsync((void**)&tau[q], np * sizeof(double), st) != cudaSuccess) {
                cudaGetLastError();
                c = YK_ERR_NO_MEMORY;
            }
        }
        if (c == YK_OK) c = yk_label(g[q], r->label_kind, r->label_param, nullptr, f[q]);
        rc[q] = c;
        if (c == YK_OK) {
            ok_g.push_back(g[q]);
            ok_f.push_back(f[q]);
            ok_s.push_back(sig[q]);
            ok_i.push_back(q);
        }
    }
    std::vector<yk_solve_info> info(ok_g.size());
    int brc = ok_g.empty() ? YK_OK
                           : solve_batch(ok_g.data(), (int)ok_g.size(), ok_f.data(), ok_s.data(),
                                         info.data());
    for (size_t t = 0; t < ok_i.size(); ++t) {
        const size_t q = ok_i[t];
        Request* r = rs[q];
        r->info = info[t];
        if (brc != YK_OK && brc != YK_ERR_NOT_CONVERGED) {
            rc[q] = brc;
            continue;
        }
        if (!(info[t].rel_residual <= r->prm.gmres_tol)) r->error = YK_ERR_NOT_CONVERGED;
        yk_geom* gg = g[q];
        double* un = gg->ws.vec[4];
        int c = normal_derivative(gg, sig[q], un, Prec::SPLIT);
        if (c == YK_OK) c = forces_torques(gg, sig[q], f[q], un, F[q], tau[q], nullptr);
        if (c == YK_OK) {
            const size_t n = (size_t)gg->n, np = (size_t)gg->np;
            r->sigma.resize(n);
            r->F.resize(2 * np);
            r->tau.resize(np);
            cudaMemcpyAsync(r->sigma.data(), sig[q], n * sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(r->F.data(), F[q], 2 * np * sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(r->tau.data(), tau[q], np * sizeof(double), cudaMemcpyDeviceToHost, st);
        }
        rc[q] = c;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess)
        for (auto& c : rc)
            if (c == YK_OK) c = YK_ERR_CUDA;
    for (size_t q = 0; q < k; ++q) {
        if (f[q]) cudaFreeAsync(f[q], st);
        if (sig[q]) cudaFreeAsync(sig[q], st);
        if (F[q]) cudaFreeAsync(F[q], st);
        if (tau[q]) cudaFreeAsync(tau[q], st);
        if (g[q]) yk_destroy_geometry(g[q]);
    }
}

// Run one request to completion on a worker's context.
static int run_request(yk_ctx* ctx, Request* r) {
    yk_geom* g = nullptr;
    int rc = yk_create_geometry(ctx, r->parts.data(), (int)r->parts.size(), &r->prm, &g);
    if (rc != YK_OK) return rc;
    const size_t n = (size_t)g->n;
    double *f = nullptr, *sig = nullptr, *F = nullptr, *tau = nullptr;
    cudaStream_t st = ctx->stream;
    if (cudaMallocAsync((void**)&f, n * sizeof(double), st) != cudaSuccess ||
        cudaMallocAsync((void**)&sig, n * sizeof(double), st) != cudaSuccess ||
        cudaMallocAsync((void**)&F, 2 * g->np * sizeof(double), st) != cudaSuccess ||
        cudaMallocAsync((void**)&tau, g->np * sizeof(double), st) != cudaSuccess) {
        cudaGetLastError();
        rc = YK_ERR_NO_MEMORY;
    }
    if (rc == YK_OK) rc = yk_label(g, r->label_kind, r->label_param, nullptr, f);
    if (rc == YK_OK) {
        rc = yk_solve_forces(g, f, sig, F, tau, &r->info);
        if (rc == YK_ERR_NOT_CONVERGED) r->error = rc, rc = YK_OK;
    }
    if (rc == YK_OK) {
        r->sigma.resize(n);
        r->F.resize(2 * g->np);
        r->tau.resize(g->np);
        cudaMemcpyAsync(r->sigma.data(), sig, n * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(r->F.data(), F, 2 * g->np * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(r->tau.data(), tau, g->np * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = YK_ERR_CUDA;
    }
    if (f) cudaFreeAsync(f, st);
    if (sig) cudaFreeAsync(sig, st);
    if (F) cudaFreeAsync(F, st);
    if (tau) cudaFreeAsync(tau, st);
    yk_destroy_geometry(g);
    return rc;
}

// The oldest queued request, if it fits the memory left (arrival order is
// kept: later requests do not overtake it). A request too large for the
// budget on its own is admitted when nothing else runs.
static Request* admit(Server* s) {
    if (s->queue.empty()) return nullptr;
    Request* r = s->reqs[s->queue.front()].get();
    if (s->mem_in_flight + r->mem_bytes <= s->mem_budget || s->running == 0) {
        s->queue.pop_front();
        return r;
    }
    return nullptr;
}

static void worker_main(Server* s) {
    cudaSetDevice(s->device);
    keep_pool_memory(s->device);
    int prio_low = 0, prio_high = 0;
    cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    cudaStream_t st_hi = nullptr, st_lo = nullptr;
    cudaStreamCreateWithPriority(&st_hi, cudaStreamNonBlocking, prio_high);
    cudaStreamCreateWithPriority(&st_lo, cudaStreamNonBlocking, prio_low);
    yk_ctx ctx;
    ctx.device = s->device;
    ctx.stream = st_lo;
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        Request* r = nullptr;
        s->cv_work.wait(lk, [&] { return s->stop || (r = admit(s)) != nullptr; });
        if (!r) break;   // stop requested and nothing admitted
        // a small batchable request takes the batchable ones queued right
        // behind it along (arrival order kept, memory permitting)
        std::vector<Request*> batch{r};
        if (batchable(r)) {
            while ((int)batch.size() < MAX_BATCH && !s->queue.empty()) {
                Request* q = s->reqs[s->queue.front()].get();
                if (!batchable(q)) break;
                const size_t mem = s->mem_in_flight + r->mem_bytes;
                size_t extra = 0;
                for (size_t b = 1; b < batch.size(); ++b) extra += batch[b]->mem_bytes;
                if (mem + extra + q->mem_bytes > s->mem_budget) break;
                s->queue.pop_front();
                batch.push_back(q);
            }
        }
        for (Request* q : batch) {
            q->status = YK_REQ_RUNNING;
            s->mem_in_flight += q->mem_bytes;
            s->running++;
        }
        lk.unlock();
        std::vector<int> rcs(batch.size(), YK_OK);
        if (batch.size() > 1) {
            ctx.stream = st_hi;
            run_batch(&ctx, batch, rcs);
        } else {
            ctx.stream = request_nodes(r) <= SMALL_REQUEST_NODES ? st_hi : st_lo;
            rcs[0] = run_request(&ctx, r);
        }
        lk.lock();
        for (size_t b = 0; b < batch.size(); ++b) {
            Request* q = batch[b];
            q->t_done = Clock::now();
            s->mem_in_flight -= q->mem_bytes;
            s->running--;
            s->finished++;
            if (rcs[b] != YK_OK) {
                q->status = YK_REQ_FAILED;
                q->error = rcs[b];
            } else {
                q->status = YK_REQ_DONE;
            }
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    lk.unlock();
    while (!ctx.geoms.empty()) yk_destroy_geometry(*ctx.geoms.begin());
    cudaStreamSynchronize(st_hi);
    cudaStreamSynchronize(st_lo);
    if (ctx.h_status) cudaFreeHost(ctx.h_status);
    ctx.h_status = nullptr;
    cudaStreamDestroy(st_hi);
    cudaStreamDestroy(st_lo);
}

static int server_of(yk_ctx* ctx, Server** out) {
    if (!ctx->server) {
        YK_TRY_CUDA(cudaSetDevice(ctx->device));
        size_t free_b = 0, total_b = 0;
        YK_TRY_CUDA(cudaMemGetInfo(&free_b, &total_b));
        auto* s = new (std::nothrow) Server();
        if (!s) return YK_ERR_NO_MEMORY;
        s->device = ctx->device;
        s->mem_budget = (size_t)(0.6 * (double)free_b);
        const int nslots = 8;
        for (int k = 0; k < nslots; ++k) s->workers.emplace_back(worker_main, s);
        ctx->server = s;
    }
    *out = (Server*)ctx->server;
    return YK_OK;
}

int destroy_server(yk_ctx* ctx) {
    if (!ctx || !ctx->server) return YK_OK;
    Server* s = (Server*)ctx->server;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->queue.clear();   // pending requests are dropped; running ones finish
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
    ctx->server = nullptr;
    return YK_OK;
}

}  // namespace yk

using namespace yk;

extern "C" {

int yk_submit(yk_ctx* ctx, const yk_particle* particles, int n_particles, const yk_params* prm,
              int label_kind, double label_param, uint64_t* request_id) {
    if (!ctx || !particles || n_particles < 1 || !prm || !request_id) return YK_ERR_ARG;
    if (label_kind < YK_LABEL_TANH || label_kind > YK_LABEL_COS) return YK_ERR_ARG;
    Server* s = nullptr;
    YK_TRY(server_of(ctx, &s));
    auto r = std::make_unique<Request>();
    r->parts.assign(particles, particles + n_particles);
    r->prm = *prm;
    r->label_kind = label_kind;
    r->label_param = label_param;
    r->mem_bytes = request_bytes(*r);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->queue.size() >= s->max_queue) return YK_ERR_BUSY;
        r->id = s->next_id++;
        *request_id = r->id;
        s->queue.push_back(r->id);
        s->reqs[r->id] = std::move(r);
    }
    s->cv_work.notify_one();
    return YK_OK;
}

int yk_poll(yk_ctx* ctx, uint64_t id, int* status, double* sigma, double* F, double* tau,
            yk_solve_info* info, double* latency_ms) {
    if (!ctx || !status) return YK_ERR_ARG;
    if (!ctx->server) return YK_ERR_NOT_FOUND;
    Server* s = (Server*)ctx->server;
    std::unique_ptr<Request> done;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) return YK_ERR_NOT_FOUND;
        *status = it->second->status;
        if (*status == YK_REQ_DONE || *status == YK_REQ_FAILED) {
            done = std::move(it->second);
            s->reqs.erase(it);
        }
    }
    if (done) {
        if (done->status == YK_REQ_DONE) {
            if (sigma) memcpy(sigma, done->sigma.data(), done->sigma.size() * sizeof(double));
            if (F) memcpy(F, done->F.data(), done->F.size() * sizeof(double));
            if (tau) memcpy(tau, done->tau.data(), done->tau.size() * sizeof(double));
            if (info) *info = done->info;
        }
        if (latency_ms)
            *latency_ms = std::chrono::duration<double, std::milli>(done->t_done - done->t_submit)
                              .count();
        if (done->error != YK_OK && done->error != YK_ERR_NOT_CONVERGED) return done->error;
    }
    return YK_OK;
}

constexpr auto DRAIN_STALL = std::chrono::minutes(5);

int yk_drain(yk_ctx* ctx) {
    if (!ctx) return YK_ERR_ARG;
    if (!ctx->server) return YK_OK;
    Server* s = (Server*)ctx->server;
    std::unique_lock<std::mutex> lk(s->mu);
    // bounded by progress: give up when no request has completed for
    // DRAIN_STALL (a request larger than the serving stream's largest takes
    // a few seconds), however long the whole queue takes
    while (!(s->queue.empty() && s->running == 0)) {
        const uint64_t seen = s->finished;
        const bool moved = s->cv_done.wait_for(lk, DRAIN_STALL, [&] {
            return s->finished != seen || (s->queue.empty() && s->running == 0);
        });
        if (!moved) return YK_ERR_TIMEOUT;
    }
    for (auto& kv : s->reqs)
        if (kv.second->status == YK_REQ_FAILED) return kv.second->error;
    return YK_OK;
}

}  // extern "C"
