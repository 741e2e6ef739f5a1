// C ABI entry points (include/yk.h): argument checking, host/device
// pointer staging, and the order of the steps of one solve (Algorithm 1,
// steps 2-6 restricted to the screened-Laplace part).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <tuple>

#include <vector>

#include "yk_internal.cuh"

namespace yk {

static thread_local char g_last_cuda[256] = "";
static std::atomic<unsigned long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_last_cuda, sizeof(g_last_cuda), "CUDA error %d (%s) in %s at %s:%d", (int)e,
             cudaGetErrorString(e), what, file, line);
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory that lives on `device` itself (managed memory counts for
// any device). Used where a pointer on another GPU would otherwise pass and
// be read through peer access or fail only in a later call.
static bool is_device_ptr_on(const void* p, int device) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

int dev_alloc(void** p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (bytes == 0) return YK_OK;
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? YK_ERR_NO_MEMORY : YK_ERR_CUDA;
    }
    return YK_OK;
}

void dev_free(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

// Pinned host mirror of the solver status, one per context (allocated on
// first use, released by yk_destroy).
double* host_status(yk_ctx* ctx) {
    if (!ctx->h_status) {
        if (cudaMallocHost((void**)&ctx->h_status, 8 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            ctx->h_status = nullptr;
        }
    }
    return ctx->h_status;
}

// Keep freed stream-ordered memory in this process's default pool of the
// device instead of returning it at every synchronisation.
void keep_pool_memory(int device) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
}

// A caller array seen from the device: the pointer itself when it is device
// memory, else a stream-ordered temporary (copied in for inputs, copied
// back by finish() for outputs).
struct Arg {
    yk_geom* g = nullptr;
    void* user = nullptr;
    void* dev = nullptr;
    size_t bytes = 0;
    bool tmp = false;
    bool out = false;
    ~Arg() {
        if (tmp && dev) cudaFreeAsync(dev, g->ctx->stream);
    }
    int init(yk_geom* gg, const void* p, size_t nbytes, bool is_out) {
        g = gg;
        user = const_cast<void*>(p);
        bytes = nbytes;
        out = is_out;
        if (!p) return YK_OK;
        if (is_device_ptr(p)) {
            dev = user;
            return YK_OK;
        }
        tmp = true;
        YK_TRY_CUDA(cudaMallocAsync(&dev, nbytes, g->ctx->stream));
        if (!is_out)
            YK_TRY_CUDA(cudaMemcpyAsync(dev, p, nbytes, cudaMemcpyHostToDevice, g->ctx->stream));
        return YK_OK;
    }
    int finish() {
        if (tmp && out && user)
            YK_TRY_CUDA(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, g->ctx->stream));
        return YK_OK;
    }
    double* d() const { return (double*)dev; }
};

static int sync(yk_geom* g) {
    YK_TRY_CUDA(cudaStreamSynchronize(g->ctx->stream));
    return YK_OK;
}

static int check_params(const yk_params* p) {
    if (!p) return YK_ERR_ARG;
    if (!(p->rho > 0.0) || !isfinite(p->rho) || !isfinite(p->gamma)) return YK_ERR_ARG;
    if (p->n_panels < 1 || p->n_gl < 2 || p->n_gl > MAX_NGL) return YK_ERR_ARG;
    if (p->qbx_order < 0 || p->qbx_order > MAX_ORDER) return YK_ERR_ARG;
    if (p->oversample < 1 || p->oversample > MAX_OVERSAMPLE) return YK_ERR_ARG;
    if (!(p->qbx_r_factor > 0.0) || p->qbx_r_factor > 1.0) return YK_ERR_ARG;
    if (p->near_width < 0) return YK_ERR_ARG;
    const int nn = (2 * p->near_width + 1 >= p->n_panels) ? p->n_panels : 2 * p->near_width + 1;
    if (nn > MAX_NEAR_PANELS) return YK_ERR_ARG;
    if (p->gmres_restart < 1 || p->gmres_restart > 1000 || p->max_iter < 1) return YK_ERR_ARG;
    if (p->precision != YK_FP64 && p->precision != YK_MIXED) return YK_ERR_ARG;
    if (!(p->gmres_tol > 0.0) || !(p->inner_tol > 0.0) || p->inner_tol >= 1.0) return YK_ERR_ARG;
    if (p->max_refine < 1) return YK_ERR_ARG;
    if (p->farfield != YK_FARFIELD_DENSE && p->farfield != YK_FARFIELD_CUTOFF &&
        p->farfield != YK_FARFIELD_FMM)
        return YK_ERR_ARG;
    if (p->fmm_order < 2 || p->fmm_order > FMM_PMAX) return YK_ERR_ARG;
    if (!(p->fmm_leaf >= 0.0) || !isfinite(p->fmm_leaf)) return YK_ERR_ARG;
    if (!(p->cutoff_tol > 0.0)) return YK_ERR_ARG;
    if (p->precond != YK_PRECOND_NONE && p->precond != YK_PRECOND_BLOCK) return YK_ERR_ARG;
    if (p->precond == YK_PRECOND_BLOCK && (int64_t)p->n_panels * p->n_gl > 1024) return YK_ERR_ARG;
    if (!(p->split_tol > 0.0) || !(p->grad_split_tol > 0.0)) return YK_ERR_ARG;
    if (p->representation != YK_REP_DOUBLE_LAYER && p->representation != YK_REP_COMBINED)
        return YK_ERR_ARG;
    if (!(p->viscosity > 0.0) || !isfinite(p->viscosity)) return YK_ERR_ARG;
    if (p->coarse != YK_COARSE_NONE && p->coarse != YK_COARSE_MODES) return YK_ERR_ARG;
    if (p->representation == YK_REP_COMBINED &&
        (p->precision != YK_FP64 || p->farfield == YK_FARFIELD_FMM || !(p->bw_eta > 0.0) ||
         !isfinite(p->bw_eta)))
        return YK_ERR_ARG;
    return YK_OK;
}

// Smallest surface gap g such that every source particle at gap >= g has
// an FP32 far-field error bound below split_tol * max|sigma|. Bound per
// source particle: eps(z) * L/(2 pi rho) * K1(z) (1 + 2/z) with z = g/rho,
// K1(z) <= sqrt(pi/(2z)) e^{-z} (1 + 1/z), and the FP32 per-pair relative
// error model eps(z) = 4e-7 (4 + 2 z + 2 R/rho) (fitted K1, exp2 argument
// rounding, FP32 coordinate rounding at distance ~ g + 2R).
// Smallest surface gap beyond which a whole source particle's contribution
// (value or normal derivative) is below tol * max|sigma|:
// L/(2 pi rho) K1(z) (1 + 2/z) * 2 with the same K1 bound, z = gap/rho.
double cutoff_gap(double rho, double perim, double tol) {
    auto bound = [&](double z) {
        const double k1ub = sqrt(PI / (2.0 * z)) * exp(-z) * (1.0 + 1.0 / z);
        return perim / (2.0 * PI * rho) * k1ub * (1.0 + 2.0 / z) * 2.0;
    };
    double lo = 0.5, hi = 4000.0;
    if (bound(hi) > tol) return INFINITY;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (bound(mid) > tol) lo = mid;
        else hi = mid;
    }
    return hi * rho;
}

static double split_gap(double rho, double perim, double rmax, double tol) {
    auto bound = [&](double z) {
        const double k1ub = sqrt(PI / (2.0 * z)) * exp(-z) * (1.0 + 1.0 / z);
        const double eps = 4e-7 * (4.0 + 2.0 * z + 2.0 * rmax / rho);
        return eps * perim / (2.0 * PI * rho) * k1ub * (1.0 + 2.0 / z) * 4.0;
    };
    double lo = 0.5, hi = 2000.0;
    if (bound(hi) > tol) return INFINITY;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (bound(mid) > tol) lo = mid;
        else hi = mid;
    }
    return hi * rho;
}

}  // namespace yk

using namespace yk;

yk::GeomView yk_geom::view() const {
    GeomView v;
    v.np = np;
    v.npan = npan;
    v.ngl = ngl;
    v.npp = npp;
    v.n = n;
    v.near_w = prm.near_width;
    v.n_near = n_near;
    v.rho = prm.rho;
    v.part = d_part;
    v.c32 = d_c32;
    v.r32 = d_r32;
    v.shape_of = d_shape_of;
    v.x = d_x;
    v.y = d_y;
    v.nx = d_nx;
    v.ny = d_ny;
    v.w = d_w;
    v.speed = d_speed;
    v.xi = d_xi;
    v.cval = d_cval;
    v.cgrad = d_cgrad;
    v.eta = prm.representation == YK_REP_COMBINED ? prm.bw_eta : 0.0;
    return v;
}

extern "C" {

int yk_default_params(yk_params* p) {
    if (!p) return YK_ERR_ARG;
    memset(p, 0, sizeof(*p));
    p->rho = 1.0;
    p->gamma = 1.0;
    p->n_panels = 16;
    p->n_gl = 16;
    p->qbx_order = 10;
    p->oversample = 8;
    p->qbx_r_factor = 0.125;
    p->near_width = 1;
    p->gmres_restart = 100;
    p->max_iter = 300;
    p->precision = YK_MIXED;
    p->gmres_tol = 1e-12;
    p->inner_tol = 1e-6;
    p->max_refine = 8;
    p->farfield = YK_FARFIELD_DENSE;
    p->split_tol = 1e-14;
    p->grad_split_tol = 1e-13;
    p->cutoff_tol = 1e-15;
    p->precond = YK_PRECOND_BLOCK;
    p->fmm_order = 12;
    p->fmm_leaf = 0.0;
    p->representation = YK_REP_DOUBLE_LAYER;
    p->bw_eta = 0.25;
    p->viscosity = 1.0;
    p->coarse = YK_COARSE_MODES;
    return YK_OK;
}

const char* yk_strerror(int code) {
    switch (code) {
        case YK_OK: return "ok";
        case YK_ERR_ARG: return "invalid argument";
        case YK_ERR_BAD_GEOMETRY: return "particles overlap";
        case YK_ERR_NO_MEMORY: return "out of device or host memory";
        case YK_ERR_NOT_CONVERGED: return "solver did not reach the tolerance";
        case YK_ERR_TIMEOUT: return "a bounded device wait gave up";
        case YK_ERR_CUDA: return g_last_cuda[0] ? g_last_cuda : "CUDA runtime error";
        case YK_ERR_NOT_FOUND: return "unknown request id";
        case YK_ERR_BUSY: return "serving queue full";
        case YK_ERR_TOO_LARGE:
            return "request exceeds the fixed scratch of the allocation-free entry point";
        default: return "unknown error code";
    }
}

int yk_create(yk_ctx** ctx, int device, void* cuda_stream) {
    if (!ctx) return YK_ERR_ARG;
    *ctx = nullptr;
    int ndev = 0;
    YK_TRY_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return YK_ERR_ARG;
    YK_TRY_CUDA(cudaSetDevice(device));
    yk_ctx* c = new (std::nothrow) yk_ctx();
    if (!c) return YK_ERR_NO_MEMORY;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    keep_pool_memory(device);
    *ctx = c;
    return YK_OK;
}

int yk_destroy(yk_ctx* ctx) {
    if (!ctx) return YK_ERR_ARG;
    destroy_server(ctx);
    while (!ctx->geoms.empty()) yk_destroy_geometry(*ctx->geoms.begin());
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->h_batch) cudaFreeHost(ctx->h_batch);
    delete ctx;
    return YK_OK;
}

int yk_destroy_geometry(yk_geom* g) {
    if (!g) return YK_ERR_ARG;
    g->ctx->geoms.erase(g);
    cudaSetDevice(g->ctx->device);
    cudaStreamSynchronize(g->ctx->stream);
    free_workspace(g);
    cudaStream_t st = g->ctx->stream;
    for (auto& L : g->lists) dev_free(L.d, st);
    for (auto& L : g->sym) dev_free(L.d, st);
    dev_free(g->nbr_off, st);
    dev_free(g->nbr, st);
    fmm_free(g);
    dyn_free(g);
    stokes_free(g);
    contact_free(g);
    coarse_free(g);
    for (auto& B : g->bands) {
        dev_free(B.off, st);
        dev_free(B.idx, st);
    }
    dev_free(g->d_counts, st);
    dev_free(g->d_mpole, st);
    dev_free(g->d_local, st);
    void* bufs[] = {g->d_part, g->d_c32, g->d_r32, g->d_counter, g->d_shape_of, g->d_shape_ab, g->d_x, g->d_y, g->d_nx, g->d_ny,
                    g->d_w, g->d_speed, g->d_xi, g->d_cval, g->d_cgrad, g->d_glx, g->d_glw,
                    g->d_interp, g->d_diff, g->d_fine_x, g->d_fine_w, g->d_minv, g->d_minv32,
                    g->d_self, g->d_self_grad, g->d_self32, g->d_particles};
    for (void* b : bufs) dev_free(b, st);
    cudaStreamSynchronize(st);
    delete g;
    return YK_OK;
}

int yk_create_geometry(yk_ctx* ctx, const yk_particle* particles, int n_particles,
                       const yk_params* prm, yk_geom** out) {
    if (!ctx || !particles || !out || n_particles < 1) return YK_ERR_ARG;
    *out = nullptr;
    YK_TRY(check_params(prm));
    const int64_t npp = (int64_t)prm->n_panels * prm->n_gl;
    const int64_t n = npp * n_particles;
    if (npp > (1 << 20) || n > ((int64_t)1 << 31)) return YK_ERR_ARG;
    // particles: valid shapes, and no certain overlap (inscribed circles)
    std::map<std::tuple<int, double, double>, int> shapes;
    std::vector<int> shape_of(n_particles);
    std::vector<double2> shape_ab;
    double rmax = 0.0;
    for (int i = 0; i < n_particles; ++i) {
        const yk_particle& P = particles[i];
        if (P.shape != YK_SHAPE_DISK && P.shape != YK_SHAPE_ELLIPSE) return YK_ERR_ARG;
        if (!(P.A > 0.0) || !(P.B > 0.0) || !isfinite(P.A) || !isfinite(P.B) ||
            !isfinite(P.cx) || !isfinite(P.cy) || !isfinite(P.phi))
            return YK_ERR_ARG;
        const double B = (P.shape == YK_SHAPE_DISK) ? P.A : P.B;
        auto key = std::make_tuple((int)P.shape, P.A, B);
        auto it = shapes.find(key);
        if (it == shapes.end()) {
            int idx = (int)shape_ab.size();
            shapes[key] = idx;
            shape_ab.push_back(make_double2(P.A, B));
            shape_of[i] = idx;
        } else {
            shape_of[i] = it->second;
        }
        rmax = std::max(rmax, std::max(P.A, B));
    }
    {
        // grid hash on inscribed radii: centres closer than rmin_i + rmin_j overlap for sure
        const double cell = 2.0 * rmax;
        std::map<std::pair<long, long>, std::vector<int>> grid;
        for (int i = 0; i < n_particles; ++i) {
            const yk_particle& P = particles[i];
            long gx = (long)floor(P.cx / cell), gy = (long)floor(P.cy / cell);
            const double ri = std::min(P.A, P.shape == YK_SHAPE_DISK ? P.A : P.B);
            for (long dx = -1; dx <= 1; ++dx)
                for (long dy = -1; dy <= 1; ++dy) {
                    auto it = grid.find({gx + dx, gy + dy});
                    if (it == grid.end()) continue;
                    for (int j : it->second) {
                        const yk_particle& Q = particles[j];
                        const double rj = std::min(Q.A, Q.shape == YK_SHAPE_DISK ? Q.A : Q.B);
                        if (hypot(P.cx - Q.cx, P.cy - Q.cy) < ri + rj) return YK_ERR_BAD_GEOMETRY;
                    }
                }
            grid[{gx, gy}].push_back(i);
        }
    }
    YK_TRY_CUDA(cudaSetDevice(ctx->device));
    yk_geom* g = new (std::nothrow) yk_geom();
    if (!g) return YK_ERR_NO_MEMORY;
    g->ctx = ctx;
    g->prm = *prm;
    g->np = n_particles;
    g->npan = prm->n_panels;
    g->ngl = prm->n_gl;
    g->npp = (int)npp;
    g->n = n;
    g->n_near = (2 * prm->near_width + 1 >= prm->n_panels) ? prm->n_panels
                                                            : 2 * prm->near_width + 1;
    g->nshape = (int)shape_ab.size();
    g->parts.assign(particles, particles + n_particles);
    for (auto& P : g->parts)
        if (P.shape == YK_SHAPE_DISK) P.B = P.A;
    g->shape_of_h = shape_of;
    g->shape_ab = shape_ab;
    g->max_radius = rmax;
    double perim = 0.0;
    for (auto& s : shape_ab) {
        // Ramanujan's perimeter bound is not needed: 2 pi max(A, B) bounds it
        perim = std::max(perim, 2.0 * PI * std::max(s.x, s.y));
    }
    g->max_perimeter = perim;
    g->split_gap = split_gap(prm->rho, perim, rmax, prm->split_tol);
    g->split_gap_grad = split_gap(prm->rho, perim, rmax, prm->grad_split_tol);
    g->cutoff_gap = (prm->farfield != YK_FARFIELD_DENSE)
                        ? cutoff_gap(prm->rho, perim, prm->cutoff_tol) : INFINITY;
    // the FMM far field serves the FP32 inner operator (pairs carry ~1e-7
    // relative error), so it reaches only as far as 1e-10 of max|sigma|
    g->fmm_gap = cutoff_gap(prm->rho, perim, std::max(prm->cutoff_tol, FMM_REACH_TOL));
    // the FP64 tiles of the split operators stay inside the cut-off
    g->split_gap = std::min(g->split_gap, g->cutoff_gap);
    g->split_gap_grad = std::min(g->split_gap_grad, g->cutoff_gap);
    g->tile_gap = std::min(g->split_gap, EXPANSION_GAP_RADII * rmax);
    g->tile_gap_grad = std::min(g->split_gap_grad, EXPANSION_GAP_RADII * rmax);
    const int os = prm->oversample;
    const size_t N = (size_t)n;
    const size_t rowlen = (size_t)g->n_near * g->ngl;
    int rc = YK_OK;
#define ALLOC(ptr, count) \
    if (rc == YK_OK) rc = dev_alloc((void**)&g->ptr, sizeof(*g->ptr) * (size_t)(count), ctx->stream)
    ALLOC(d_part, n_particles);
    ALLOC(d_particles, n_particles);
    ALLOC(d_c32, n_particles);
    ALLOC(d_r32, n_particles);
    ALLOC(d_counter, 1);
    ALLOC(d_counts, n_particles);
    ALLOC(d_mpole, (size_t)n_particles * EXPANSION_TERMS);
    ALLOC(d_local, (size_t)n_particles * EXPANSION_TERMS);
    ALLOC(d_shape_of, n_particles);
    ALLOC(d_shape_ab, g->nshape);
    ALLOC(d_x, N);
    ALLOC(d_y, N);
    ALLOC(d_nx, N);
    ALLOC(d_ny, N);
    ALLOC(d_w, N);
    ALLOC(d_speed, N);
    ALLOC(d_xi, N);
    ALLOC(d_cval, (size_t)g->nshape * npp * rowlen);
    ALLOC(d_cgrad, (size_t)g->nshape * npp * rowlen);
    g->use_self = npp <= SELF_BLOCK_MAX_NODES;
    if (g->use_self) {
        ALLOC(d_self, (size_t)g->nshape * npp * npp);
        ALLOC(d_self_grad, (size_t)g->nshape * npp * npp);
        ALLOC(d_self32, (size_t)g->nshape * npp * npp);
    }
    ALLOC(d_glx, g->ngl);
    ALLOC(d_glw, g->ngl);
    ALLOC(d_interp, (size_t)os * g->ngl * g->ngl);
    ALLOC(d_diff, (size_t)g->ngl * g->ngl);
    ALLOC(d_fine_x, (size_t)os * g->ngl);
    ALLOC(d_fine_w, (size_t)os * g->ngl);
    if (prm->precond == YK_PRECOND_BLOCK) {
        ALLOC(d_minv, (size_t)g->nshape * npp * npp);
        ALLOC(d_minv32, (size_t)g->nshape * npp * npp);
    }
#undef ALLOC
    if (rc == YK_OK) rc = alloc_workspace(g);
    if (rc == YK_OK) {
        cudaError_t e = cudaMemcpyAsync(g->d_shape_of, shape_of.data(), sizeof(int) * n_particles,
                                        cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->d_shape_ab, shape_ab.data(), sizeof(double2) * g->nshape,
                                cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) {
            set_cuda_error(e, "upload", __FILE__, __LINE__);
            rc = YK_ERR_CUDA;
        }
    }
    if (rc == YK_OK) rc = build_geometry(g);
    ctx->geoms.insert(g);
    if (rc != YK_OK) {
        yk_destroy_geometry(g);
        return rc;
    }
    *out = g;
    return YK_OK;
}

int yk_update_geometry(yk_geom* g, const yk_particle* particles, int n_particles) {
    if (!g || !particles || n_particles != g->np) return YK_ERR_ARG;
    for (int i = 0; i < n_particles; ++i) {
        const yk_particle& P = particles[i];
        const yk_particle& Q = g->parts[i];
        const double B = (P.shape == YK_SHAPE_DISK) ? P.A : P.B;
        if (P.shape != Q.shape || P.A != Q.A || B != Q.B) return YK_ERR_ARG;
        if (!isfinite(P.cx) || !isfinite(P.cy) || !isfinite(P.phi)) return YK_ERR_ARG;
    }
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    for (int i = 0; i < n_particles; ++i) {
        g->parts[i].cx = particles[i].cx;
        g->parts[i].cy = particles[i].cy;
        g->parts[i].phi = particles[i].phi;
    }
    return update_nodes(g);
}

int yk_kernel_launches(uint64_t* count) {
    if (!count) return YK_ERR_ARG;
    *count = g_launches.load(std::memory_order_relaxed);
    return YK_OK;
}

int yk_num_nodes(const yk_geom* g, int64_t* n) {
    if (!g || !n) return YK_ERR_ARG;
    *n = g->n;
    return YK_OK;
}

int yk_nodes(const yk_geom* g, double* xy, double* nrm, double* w) {
    if (!g) return YK_ERR_ARG;
    yk_geom* gg = const_cast<yk_geom*>(g);
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    const size_t N = (size_t)g->n;
    auto pair_out = [&](double* dst, const double* a, const double* b) -> int {
        if (!dst) return YK_OK;
        Arg o;
        YK_TRY(o.init(gg, dst, 2 * N * sizeof(double), true));
        YK_TRY_CUDA(cudaMemcpy2DAsync(o.d(), 2 * sizeof(double), a, sizeof(double), sizeof(double),
                                      N, cudaMemcpyDeviceToDevice, st));
        YK_TRY_CUDA(cudaMemcpy2DAsync(o.d() + 1, 2 * sizeof(double), b, sizeof(double),
                                      sizeof(double), N, cudaMemcpyDeviceToDevice, st));
        YK_TRY(o.finish());
        return sync(gg);
    };
    YK_TRY(pair_out(xy, g->d_x, g->d_y));
    YK_TRY(pair_out(nrm, g->d_nx, g->d_ny));
    if (w) {
        YK_TRY_CUDA(cudaMemcpyAsync(w, g->d_w, N * sizeof(double), cudaMemcpyDefault, st));
        YK_TRY(sync(gg));
    }
    return YK_OK;
}

int yk_label(yk_geom* g, int kind, double param, const double* f_custom, double* f_out) {
    if (!g || !f_out) return YK_ERR_ARG;
    if (kind < YK_LABEL_TANH || kind > YK_LABEL_CUSTOM) return YK_ERR_ARG;
    if (kind == YK_LABEL_CUSTOM && !f_custom) return YK_ERR_ARG;
    if (kind == YK_LABEL_SINP && (param < 0 || param > 64 || param != floor(param)))
        return YK_ERR_ARG;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    const size_t bytes = (size_t)g->n * sizeof(double);
    Arg o;
    YK_TRY(o.init(g, f_out, bytes, true));
    if (kind == YK_LABEL_CUSTOM) {
        YK_TRY_CUDA(cudaMemcpyAsync(o.d(), f_custom, bytes, cudaMemcpyDefault, g->ctx->stream));
    } else {
        YK_TRY(launch_label(g, kind, param, o.d()));
    }
    YK_TRY(o.finish());
    return sync(g);
}

int yk_matvec(yk_geom* g, const double* sigma, double* y, int precision) {
    if (!g || !sigma || !y) return YK_ERR_ARG;
    if (precision != YK_FP64 && precision != YK_MIXED) return YK_ERR_ARG;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    const size_t bytes = (size_t)g->n * sizeof(double);
    Arg a, o;
    YK_TRY(a.init(g, sigma, bytes, false));
    YK_TRY(o.init(g, y, bytes, true));
    YK_TRY(matvec(g, a.d(), o.d(), precision == YK_FP64 ? Prec::F64 : Prec::F32));
    YK_TRY(o.finish());
    return sync(g);
}

int yk_normal_derivative(yk_geom* g, const double* sigma, double* u_nu, int precision) {
    if (!g || !sigma || !u_nu) return YK_ERR_ARG;
    if (precision != YK_FP64 && precision != YK_MIXED) return YK_ERR_ARG;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    const size_t bytes = (size_t)g->n * sizeof(double);
    Arg a, o;
    YK_TRY(a.init(g, sigma, bytes, false));
    YK_TRY(o.init(g, u_nu, bytes, true));
    YK_TRY(normal_derivative(g, a.d(), o.d(), precision == YK_FP64 ? Prec::F64 : Prec::SPLIT));
    YK_TRY(o.finish());
    return sync(g);
}

int yk_solve(yk_geom* g, const double* f, double* sigma, const double* sigma0,
             yk_solve_info* info) {
    if (!g || !f || !sigma) return YK_ERR_ARG;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    const size_t bytes = (size_t)g->n * sizeof(double);
    Arg a, o, s0;
    YK_TRY(a.init(g, f, bytes, false));
    YK_TRY(s0.init(g, sigma0, bytes, false));
    YK_TRY(o.init(g, sigma, bytes, true));
    int rc = solve(g, a.d(), o.d(), sigma0 ? s0.d() : nullptr, info);
    if (rc != YK_OK && rc != YK_ERR_NOT_CONVERGED) return rc;
    YK_TRY(o.finish());
    YK_TRY(sync(g));
    return rc;
}

int yk_solve_batch(yk_geom* const* geoms, int count, const double* const* f,
                   double* const* sigma, yk_solve_info* info) {
    if (!geoms || !f || !sigma || count < 0) return YK_ERR_ARG;
    if (count == 0) return YK_OK;
    for (int s = 0; s < count; ++s)
        if (!geoms[s] || !f[s] || !sigma[s] || geoms[s]->ctx != geoms[0]->ctx) return YK_ERR_ARG;
    for (int s = 0; s < count; ++s)
        for (int t = 0; t < s; ++t)
            if (geoms[s] == geoms[t]) return YK_ERR_ARG;   // one workspace per system
    YK_TRY_CUDA(cudaSetDevice(geoms[0]->ctx->device));
    std::vector<Arg> a(count), o(count);
    std::vector<const double*> fd(count);
    std::vector<double*> sd(count);
    for (int s = 0; s < count; ++s) {
        const size_t bytes = (size_t)geoms[s]->n * sizeof(double);
        YK_TRY(a[s].init(geoms[s], f[s], bytes, false));
        YK_TRY(o[s].init(geoms[s], sigma[s], bytes, true));
        fd[s] = a[s].d();
        sd[s] = o[s].d();
    }
    const int rc = solve_batch(geoms, count, fd.data(), sd.data(), info);
    if (rc != YK_OK && rc != YK_ERR_NOT_CONVERGED) return rc;
    for (int s = 0; s < count; ++s) YK_TRY(o[s].finish());
    YK_TRY(sync(geoms[0]));
    return rc;
}

int yk_forces_torques(yk_geom* g, const double* sigma, const double* f, double* F, double* tau,
                      double* net) {
    if (!g || !sigma || !f || !F || !tau) return YK_ERR_ARG;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    const size_t bytes = (size_t)g->n * sizeof(double);
    Arg a, b, oF, ot, on;
    YK_TRY(a.init(g, sigma, bytes, false));
    YK_TRY(b.init(g, f, bytes, false));
    YK_TRY(oF.init(g, F, 2 * g->np * sizeof(double), true));
    YK_TRY(ot.init(g, tau, g->np * sizeof(double), true));
    YK_TRY(on.init(g, net, 3 * sizeof(double), true));
    double* un = g->ws.vec[4];
    YK_TRY(normal_derivative(g, a.d(), un, g->prm.precision == YK_FP64 ? Prec::F64 : Prec::SPLIT));
    YK_TRY(forces_torques(g, a.d(), b.d(), un, oF.d(), ot.d(), net ? on.d() : nullptr));
    YK_TRY(oF.finish());
    YK_TRY(ot.finish());
    YK_TRY(on.finish());
    return sync(g);
}

int yk_repulsion(yk_geom* g, double c0, int q, double* F, double* tau, double* phi) {
    if (!g || !(c0 >= 0.0) || !isfinite(c0) || q < 1 || q > 16) return YK_ERR_ARG;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    Arg oF, ot, op;
    YK_TRY(oF.init(g, F, 2 * g->np * sizeof(double), true));
    YK_TRY(ot.init(g, tau, g->np * sizeof(double), true));
    YK_TRY(op.init(g, phi, g->np * sizeof(double), true));
    double* scratch = nullptr;
    YK_TRY_CUDA(cudaMallocAsync((void**)&scratch, sizeof(double) * 4 * g->np, g->ctx->stream));
    int rc = repulsion_host(g, c0, q, F ? oF.d() : scratch, tau ? ot.d() : scratch + 2 * g->np,
                            phi ? op.d() : scratch + 3 * g->np);
    if (rc == YK_OK) rc = oF.finish();
    if (rc == YK_OK) rc = ot.finish();
    if (rc == YK_OK) rc = op.finish();
    cudaFreeAsync(scratch, g->ctx->stream);
    YK_TRY(rc);
    return sync(g);
}

int yk_default_dynamics(yk_dynamics* d) {
    if (!d) return YK_ERR_ARG;
    memset(d, 0, sizeof(*d));
    d->dt = 0.1;
    d->xi_x = 4.0 * PI;
    d->xi_theta = 4.0 * PI;
    d->c0 = 0.01;
    d->q = 3;
    d->label_kind = YK_LABEL_TANH;
    d->label_param = 10.0;
    d->warm_start = 1;
    d->mobility = 0;
    return YK_OK;
}

int yk_step(yk_geom* g, const yk_dynamics* d, int n_steps, yk_particle* particles,
            double* energy, yk_solve_info* info) {
    if (!g || !d || n_steps < 0) return YK_ERR_ARG;
    if (!(d->dt >= 0.0) || !(d->xi_x > 0.0) || !(d->xi_theta > 0.0) || !(d->c0 >= 0.0) ||
        !isfinite(d->dt) || !isfinite(d->c0) || d->q < 1 || d->q > 16)
        return YK_ERR_ARG;
    if (d->label_kind != YK_LABEL_TANH && d->label_kind != YK_LABEL_SINP &&
        d->label_kind != YK_LABEL_COS)
        return YK_ERR_ARG;
    if (d->mobility != 0 && d->mobility != 1) return YK_ERR_ARG;
    if (d->mobility && (g->npan < 3 || g->npp > 512)) return YK_ERR_ARG;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    for (int s = 0; s < n_steps; ++s)
        YK_TRY(step(g, *d, info ? info + s : nullptr, energy ? energy + s : nullptr));
    if (particles) {
        if (is_device_ptr(particles))
            YK_TRY_CUDA(cudaMemcpyAsync(particles, g->parts.data(), sizeof(yk_particle) * g->np,
                                        cudaMemcpyHostToDevice, g->ctx->stream));
        else
            memcpy(particles, g->parts.data(), sizeof(yk_particle) * g->np);
    }
    return sync(g);
}

int yk_stokes_apply(yk_geom* g, int op, const double* sigma, double* out, int precision) {
    if (!g || !sigma || !out) return YK_ERR_ARG;
    if (op != YK_STOKES_TRACTION && op != YK_STOKES_COMPLETED && op != YK_STOKES_VELOCITY)
        return YK_ERR_ARG;
    if (precision != YK_FP64 && precision != YK_MIXED) return YK_ERR_ARG;
    if (g->npan < 3 || g->npp > 512) return YK_ERR_ARG;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    const size_t bytes = 2 * (size_t)g->n * sizeof(double);
    Arg a, o;
    YK_TRY(a.init(g, sigma, bytes, false));
    YK_TRY(o.init(g, out, bytes, true));
    YK_TRY(stokes_apply(g, a.d(), o.d(), precision == YK_MIXED ? Prec::F32 : Prec::F64, op));
    YK_TRY(o.finish());
    return sync(g);
}

int yk_mobility(yk_geom* g, const double* F, const double* tau, double* v, double* omega,
                double* sigma, yk_solve_info* info) {
    if (!g || !F || !tau || !v || !omega) return YK_ERR_ARG;
    if (g->npan < 3 || g->npp > 512) return YK_ERR_ARG;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    const size_t np = (size_t)g->np;
    Arg aF, at, ov, oo, os;
    YK_TRY(aF.init(g, F, 2 * np * sizeof(double), false));
    YK_TRY(at.init(g, tau, np * sizeof(double), false));
    YK_TRY(ov.init(g, v, 2 * np * sizeof(double), true));
    YK_TRY(oo.init(g, omega, np * sizeof(double), true));
    YK_TRY(os.init(g, sigma, 2 * (size_t)g->n * sizeof(double), true));
    const int rc = mobility(g, aF.d(), at.d(), ov.d(), oo.d(), sigma ? os.d() : nullptr, info);
    if (rc != YK_OK && rc != YK_ERR_NOT_CONVERGED) return rc;
    YK_TRY(ov.finish());
    YK_TRY(oo.finish());
    YK_TRY(os.finish());
    YK_TRY(sync(g));
    return rc;
}

int yk_energy(yk_geom* g, const double* sigma, const double* f, double* phi, double* phi_total) {
    if (!g || !sigma || !f || (!phi && !phi_total)) return YK_ERR_ARG;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    const size_t bytes = (size_t)g->n * sizeof(double);
    Arg a, b, op, ot;
    YK_TRY(a.init(g, sigma, bytes, false));
    YK_TRY(b.init(g, f, bytes, false));
    YK_TRY(ot.init(g, phi_total, sizeof(double), true));
    double* un = g->ws.vec[4];
    double* ph = g->ws.vec[3];          // per-particle parts when the caller wants none
    if (phi) {
        YK_TRY(op.init(g, phi, g->np * sizeof(double), true));
        ph = op.d();
    }
    YK_TRY(normal_derivative(g, a.d(), un, g->prm.precision == YK_FP64 ? Prec::F64 : Prec::SPLIT));
    YK_TRY(energy(g, b.d(), un, ph, phi_total ? ot.d() : nullptr));
    if (phi) YK_TRY(op.finish());
    YK_TRY(ot.finish());
    return sync(g);
}

int yk_eval_potential(yk_geom* g, const double* sigma, const double* targets, int64_t nt,
                      double* u) {
    if (!g || !sigma || nt < 0 || (nt > 0 && (!targets || !u))) return YK_ERR_ARG;
    if (nt == 0) return YK_OK;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    Arg a, t, o;
    YK_TRY(a.init(g, sigma, (size_t)g->n * sizeof(double), false));
    YK_TRY(t.init(g, targets, (size_t)nt * 2 * sizeof(double), false));
    YK_TRY(o.init(g, u, (size_t)nt * sizeof(double), true));
    YK_TRY(potential(g, a.d(), t.d(), nt, o.d()));
    YK_TRY(o.finish());
    return sync(g);
}

int yk_eval_potential_near(yk_geom* g, const double* sigma, const double* targets, int64_t nt,
                           double* u) {
    if (!g || !sigma || nt < 0 || (nt > 0 && (!targets || !u))) return YK_ERR_ARG;
    if (g->prm.representation != YK_REP_DOUBLE_LAYER) return YK_ERR_ARG;
    if (nt == 0) return YK_OK;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    Arg a, t, o;
    YK_TRY(a.init(g, sigma, (size_t)g->n * sizeof(double), false));
    YK_TRY(t.init(g, targets, (size_t)nt * 2 * sizeof(double), false));
    YK_TRY(o.init(g, u, (size_t)nt * sizeof(double), true));
    YK_TRY(potential_near(g, a.d(), t.d(), nt, o.d()));
    YK_TRY(o.finish());
    return sync(g);
}

int yk_eval_potential_noalloc(yk_geom* g, const double* sigma, const double* targets,
                              int64_t nt, double* u) {
    if (!g || !sigma || nt < 0 || (nt > 0 && (!targets || !u))) return YK_ERR_ARG;
    if (nt == 0) return YK_OK;
    // device pointers on the context's device only: staging host arrays
    // would need allocations
    const int dev = g->ctx->device;
    if (!is_device_ptr_on(sigma, dev) || !is_device_ptr_on(targets, dev) ||
        !is_device_ptr_on(u, dev))
        return YK_ERR_ARG;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    return potential_noalloc(g, sigma, targets, nt, u);
}

int yk_solve_forces(yk_geom* g, const double* f, double* sigma, double* F, double* tau,
                    yk_solve_info* info) {
    if (!g || !f || !sigma || !F || !tau) return YK_ERR_ARG;
    YK_TRY_CUDA(cudaSetDevice(g->ctx->device));
    const size_t bytes = (size_t)g->n * sizeof(double);
    Arg a, o, oF, ot;
    YK_TRY(a.init(g, f, bytes, false));
    YK_TRY(o.init(g, sigma, bytes, true));
    YK_TRY(oF.init(g, F, 2 * g->np * sizeof(double), true));
    YK_TRY(ot.init(g, tau, g->np * sizeof(double), true));
    int rc = solve(g, a.d(), o.d(), nullptr, info);
    if (rc != YK_OK && rc != YK_ERR_NOT_CONVERGED) return rc;
    double* un = g->ws.vec[4];
    YK_TRY(normal_derivative(g, o.d(), un, g->prm.precision == YK_FP64 ? Prec::F64 : Prec::SPLIT));
    YK_TRY(forces_torques(g, o.d(), a.d(), un, oF.d(), ot.d(), nullptr));
    YK_TRY(o.finish());
    YK_TRY(oF.finish());
    YK_TRY(ot.finish());
    YK_TRY(sync(g));
    return rc;
}

}  // extern "C"
