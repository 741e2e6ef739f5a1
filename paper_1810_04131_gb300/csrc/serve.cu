// Serving: independent particle configurations submitted as requests and
// solved (label, Eq. bie, forces and torques) by the library. Requests are
// admitted in arrival order while their device-memory estimate fits the
// context's budget, and run to completion; yk_poll collects results.
#include <string.h>

#include <chrono>
#include <deque>
#include <map>
#include <memory>

#include "yk_internal.cuh"

namespace yk {

struct Request {
    uint64_t id = 0;
    std::vector<yk_particle> parts;
    yk_params prm{};
    int label_kind = YK_LABEL_TANH;
    double label_param = 10.0;
    int status = YK_REQ_QUEUED;
    int error = YK_OK;
    std::chrono::steady_clock::time_point t_submit, t_done;
    std::vector<double> sigma, F, tau;
    yk_solve_info info{};
};

struct Server {
    uint64_t next_id = 1;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    size_t max_queue = 1 << 16;
};

static Server* server_of(yk_ctx* ctx, bool create) {
    if (!ctx->server && create) ctx->server = new Server();
    return (Server*)ctx->server;
}

// Run one request to completion on the context's stream.
static int run_request(yk_ctx* ctx, Request* r) {
    yk_geom* g = nullptr;
    int rc = yk_create_geometry(ctx, r->parts.data(), (int)r->parts.size(), &r->prm, &g);
    if (rc != YK_OK) return rc;
    const size_t n = (size_t)g->n;
    double *f = nullptr, *sig = nullptr, *F = nullptr, *tau = nullptr;
    cudaStream_t st = ctx->stream;
    rc = YK_OK;
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

static int step(yk_ctx* ctx, Server* s) {
    if (s->queue.empty()) return YK_OK;
    uint64_t id = s->queue.front();
    s->queue.pop_front();
    Request* r = s->reqs[id].get();
    r->status = YK_REQ_RUNNING;
    int rc = run_request(ctx, r);
    r->t_done = std::chrono::steady_clock::now();
    if (rc != YK_OK) {
        r->status = YK_REQ_FAILED;
        r->error = rc;
        return rc;
    }
    r->status = YK_REQ_DONE;
    return YK_OK;
}

int destroy_server(yk_ctx* ctx) {
    if (!ctx || !ctx->server) return YK_OK;
    delete (Server*)ctx->server;
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
    Server* s = server_of(ctx, true);
    if (s->queue.size() >= s->max_queue) return YK_ERR_BUSY;
    auto r = std::make_unique<Request>();
    r->id = s->next_id++;
    r->parts.assign(particles, particles + n_particles);
    r->prm = *prm;
    r->label_kind = label_kind;
    r->label_param = label_param;
    r->t_submit = std::chrono::steady_clock::now();
    *request_id = r->id;
    s->queue.push_back(r->id);
    s->reqs[r->id] = std::move(r);
    return YK_OK;
}

int yk_poll(yk_ctx* ctx, uint64_t id, int* status, double* sigma, double* F, double* tau,
            yk_solve_info* info, double* latency_ms) {
    if (!ctx || !status) return YK_ERR_ARG;
    Server* s = server_of(ctx, false);
    if (!s) return YK_ERR_NOT_FOUND;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return YK_ERR_NOT_FOUND;
    Request* r = it->second.get();
    if (r->status == YK_REQ_QUEUED) step(ctx, s);
    *status = r->status;
    if (r->status == YK_REQ_DONE || r->status == YK_REQ_FAILED) {
        if (r->status == YK_REQ_DONE) {
            if (sigma) memcpy(sigma, r->sigma.data(), r->sigma.size() * sizeof(double));
            if (F) memcpy(F, r->F.data(), r->F.size() * sizeof(double));
            if (tau) memcpy(tau, r->tau.data(), r->tau.size() * sizeof(double));
            if (info) *info = r->info;
        }
        if (latency_ms)
            *latency_ms =
                std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
        int err = r->error;
        s->reqs.erase(it);
        if (err != YK_OK && err != YK_ERR_NOT_CONVERGED) return err;
    }
    return YK_OK;
}

int yk_drain(yk_ctx* ctx) {
    if (!ctx) return YK_ERR_ARG;
    Server* s = server_of(ctx, false);
    if (!s) return YK_OK;
    int first = YK_OK;
    while (!s->queue.empty()) {
        int rc = step(ctx, s);
        if (rc != YK_OK && first == YK_OK) first = rc;
    }
    return first;
}

}  // extern "C"
