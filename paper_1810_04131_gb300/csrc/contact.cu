// Near contact. When two particles come closer than the configurations' gaps,
// plain Gauss-Legendre quadrature on a panel of one particle loses accuracy at
// the nodes of the other (the kernel varies on the scale of the gap, not of
// the panel). A panel k of particle P whose nearest node is closer to a
// target node x_i of another particle than CONTACT_FACTOR x the panel's
// arclength is therefore integrated on its oversampled nodes (8 sub-panels
// of n_gl Gauss-Legendre nodes, sigma interpolated by the panel's Lagrange
// basis, as for the QBX coefficients):
//   y_i += sum_f kernel(x_i, y_f) w_f sigma_f - sum_j kernel(x_i, y_j) w_j sigma_j,
// the second sum being what the far-field evaluators already added. The
// correction runs in FP64 for every operator (value and normal derivative,
// every precision and far-field mode), so the FP32 inner operator stays
// consistent with the FP64-accurate residual near contact. At the
// configurations' gaps (>= 0.2 against a largest panel arclength of 0.39)
// nothing is flagged.
#include <math.h>

#include <algorithm>

#include "bessel.cuh"
#include "yk_internal.cuh"

namespace yk {

constexpr double CONTACT_FACTOR = 0.5;

// defined in p2p.cu: exclusive scan of n counts into off[0..n]
__global__ void k_scan_offsets(int np, const int* __restrict__ counts, int* __restrict__ off);

// Largest panel arclength over all particles (sum of node weights per panel),
// as the bits of a non-negative double raised with atomicMax.
__global__ void k_contact_hmax(GeomView G, unsigned long long* __restrict__ hbits) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // (particle, panel)
    if (q >= (int64_t)G.np * G.npan) return;
    const int64_t base = q * G.ngl;
    double h = 0.0;
    for (int j = 0; j < G.ngl; ++j) h += G.w[base + j];
    atomicMax(hbits, (unsigned long long)__double_as_longlong(h));
}

// Partners of each particle: the others whose bounding circles are closer
// than thr (at most CONTACT_MAX_PARTNERS; flag[0] = 1 beyond); flag[1]
// counts them all.
// One warp per particle Q, lanes over P; partners kept in order of P.
__global__ void k_contact_partners(int np, const d4* __restrict__ part, double thr,
                                   int* __restrict__ partners, int* __restrict__ npartners,
                                   int* __restrict__ flag) {
    const int Q = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (Q >= np) return;   // warp-uniform
    const d4 a = part[Q];
    int c = 0;
    bool full = false;
    for (int P0 = 0; P0 < np && !full; P0 += 32) {
        const int P = P0 + lane;
        bool hit = false;
        if (P < np && P != Q) {
            const d4 b = part[P];
            const double dx = a.x - b.x, dy = a.y - b.y;
            hit = sqrt(dx * dx + dy * dy) - a.z - b.z < thr;
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        const int k = c + __popc(m & ((1u << lane) - 1u));
        if (hit && k < CONTACT_MAX_PARTNERS) partners[Q * CONTACT_MAX_PARTNERS + k] = P;
        c += __popc(m);
        if (c > CONTACT_MAX_PARTNERS) {
            full = true;
            c = CONTACT_MAX_PARTNERS;
            if (lane == 0) atomicExch(&flag[0], 1);
        }
    }
    if (lane == 0) {
        npartners[Q] = c;
        if (c > 0) atomicAdd(&flag[1], c);
    }
}

// Entries of node i: (P, k) for the partners' panels closer than
// CONTACT_FACTOR x their arclength, partner by partner, panel by panel (a
// fixed order). Count pass (FILL = false) and fill pass.
template <bool FILL>
__global__ void k_contact_entries(GeomView G, const int* __restrict__ partners,
                                  const int* __restrict__ npartners, int* __restrict__ counts,
                                  const int* __restrict__ off, int2* __restrict__ ent,
                                  int* __restrict__ tgt, int* __restrict__ flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= G.n) return;
    const int Q = (int)(i / G.npp);
    const int np_ = npartners[Q];
    int c = 0;
    int64_t k0 = FILL ? off[i] : 0;
    if (np_ > 0) {
        const double xi = G.x[i], yi = G.y[i];
        for (int a = 0; a < np_; ++a) {
            const int P = partners[Q * CONTACT_MAX_PARTNERS + a];
            for (int k = 0; k < G.npan; ++k) {
                const int64_t base = (int64_t)P * G.npp + (int64_t)k * G.ngl;
                double h = 0.0, dmin = INFINITY;
                for (int j = 0; j < G.ngl; ++j) {
                    h += G.w[base + j];
                    const double dx = G.x[base + j] - xi, dy = G.y[base + j] - yi;
                    dmin = fmin(dmin, dx * dx + dy * dy);
                }
                if (sqrt(dmin) < CONTACT_FACTOR * h) {
                    if (FILL) ent[k0 + c] = make_int2(P, k);
                    ++c;
                }
            }
        }
    }
    if (!FILL) {
        counts[i] = c;
    } else if (c > 0) {
        tgt[atomicAdd(&flag[1], 1)] = (int)i;
    }
}

__device__ __forceinline__ void contact_curve(const yk_particle& p, double t, double& x,
                                              double& y, double& nx, double& ny, double& spd) {
    double s, c, sp, cp;
    sincos(t, &s, &c);
    sincos(p.phi, &sp, &cp);
    const double u = p.A * c, v = p.B * s, du = -p.A * s, dv = p.B * c;
    x = p.cx + cp * u - sp * v;
    y = p.cy + sp * u + cp * v;
    const double dx = cp * du - sp * dv, dy = sp * du + cp * dv;
    spd = sqrt(dx * dx + dy * dy);
    nx = dy / spd;
    ny = -dx / spd;
}

// The double-layer kernel (value: dG/dnu_y) or its normal derivative at the
// target (nu_x . grad_x dG/dnu_y), times 2 pi (the caller divides).
// (times 2 pi) the kernel of the operator (GRAD: its normal derivative at the
// target): dG/dnu_y, plus eta G in the combined representation.
template <bool GRAD>
__device__ __forceinline__ double contact_kernel(double dx, double dy, double nxs, double nys,
                                                 double nxt, double nyt, double rho, double eta) {
    const double r = sqrt(dx * dx + dy * dy);
    double k0v, k1v;
    k01(r / rho, k0v, k1v);
    const double dn_s = dx * nxs + dy * nys;
    if (!GRAD) return k1v * dn_s / (rho * r) + eta * k0v;
    const double gg = k1v / (rho * r);
    const double gp = -(k0v / rho + 2.0 * k1v / r) / (rho * r);
    const double dn_t = dx * nxt + dy * nyt;
    return gg * (nxt * nxs + nyt * nys) + gp * dn_s * dn_t / r - eta * k1v * dn_t / (rho * r);
}

// One warp per flagged node: oversampled minus plain quadrature of each of
// its flagged panels, added to out.
template <bool GRAD>
__global__ void __launch_bounds__(128) k_contact_apply(GeomView G,
                                                       const yk_particle* __restrict__ parts,
                                                       const double* __restrict__ sigma,
                                                       const int* __restrict__ off,
                                                       const int2* __restrict__ ent,
                                                       const int* __restrict__ tgt, int ntgt,
                                                       int os, const double* __restrict__ fine_x,
                                                       const double* __restrict__ fine_w,
                                                       const double* __restrict__ interp,
                                                       double* __restrict__ out) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= ntgt) return;
    const int64_t i = tgt[w];
    const double xi = G.x[i], yi = G.y[i], nxt = G.nx[i], nyt = G.ny[i];
    const double rho = G.rho;
    const double dt = 2.0 * PI / G.npan;
    const int nfp = os * G.ngl;
    double acc = 0.0;
    for (int e = off[i]; e < off[i + 1]; ++e) {
        const int P = ent[e].x, k = ent[e].y;
        const yk_particle p = parts[P];
        const int64_t base = (int64_t)P * G.npp + (int64_t)k * G.ngl;
        for (int m = lane; m < nfp; m += 32) {        // oversampled nodes
            double yx, yy, nx, ny, spd;
            contact_curve(p, k * dt + 0.5 * dt * (fine_x[m] + 1.0), yx, yy, nx, ny, spd);
            double sf = 0.0;
            for (int j = 0; j < G.ngl; ++j) sf = fma(interp[m * G.ngl + j], sigma[base + j], sf);
            acc += contact_kernel<GRAD>(xi - yx, yi - yy, nx, ny, nxt, nyt, rho, G.eta) *
                   (0.5 * dt * fine_w[m] * spd) * sf;
        }
        for (int j = lane; j < G.ngl; j += 32)        // minus the plain nodes
            acc -= contact_kernel<GRAD>(xi - G.x[base + j], yi - G.y[base + j], G.nx[base + j],
                                        G.ny[base + j], nxt, nyt, rho, G.eta) *
                   G.w[base + j] * sigma[base + j];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[i] += acc / (2.0 * PI);
}

static int grow_int(void** p, int64_t* cap, int64_t need, size_t elem, cudaStream_t st) {
    if (need <= *cap && *p) return YK_OK;
    dev_free(*p, st);
    *p = nullptr;
    *cap = 0;
    YK_TRY(dev_alloc(p, elem * (size_t)std::max<int64_t>(need, 1), st));
    *cap = need;
    return YK_OK;
}

// Build the lists for the current positions (on first use after a move).
static int contact_build(yk_geom* g) {
    Contact& C = g->contact;
    cudaStream_t st = g->ctx->stream;
    GeomView G = g->view();
    if (!C.partners) {
        YK_TRY(dev_alloc((void**)&C.partners, sizeof(int) * CONTACT_MAX_PARTNERS * g->np, st));
        YK_TRY(dev_alloc((void**)&C.npartners, sizeof(int) * g->np, st));
        YK_TRY(dev_alloc((void**)&C.flag, sizeof(int) * 4, st));
    }
    unsigned long long* hbits = reinterpret_cast<unsigned long long*>(C.flag + 2);
    YK_TRY_CUDA(cudaMemsetAsync(C.flag, 0, sizeof(int) * 4, st));
    YK_LAUNCH(k_contact_hmax, ceil_div((int64_t)g->np * g->npan, 256), 256, 0, st, G, hbits);
    unsigned long long hb = 0;
    YK_TRY_CUDA(cudaMemcpyAsync(&hb, hbits, sizeof(hb), cudaMemcpyDeviceToHost, st));
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    double hmax;
    memcpy(&hmax, &hb, sizeof(double));
    YK_LAUNCH(k_contact_partners, ceil_div(g->np, 4), 128, 0, st, g->np, g->d_part,
              CONTACT_FACTOR * hmax, C.partners, C.npartners, C.flag);
    int hf[2] = {0, 0};
    YK_TRY_CUDA(cudaMemcpyAsync(hf, C.flag, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    if (hf[0]) return YK_ERR_BAD_GEOMETRY;    // more particles in contact than supported
    C.ntgt = 0;
    if (hf[1] > 0) {        // most configurations have no partners and build no lists
        if (!C.off) {
            YK_TRY(dev_alloc((void**)&C.off, sizeof(int) * (g->n + 1), st));
            YK_TRY(dev_alloc((void**)&C.tgt, sizeof(int) * g->n, st));
        }
        int* counts = reinterpret_cast<int*>(g->ws.partial);   // >= n doubles of scratch
        YK_LAUNCH(k_contact_entries<false>, ceil_div(g->n, 256), 256, 0, st, G, C.partners,
                  C.npartners, counts, (const int*)nullptr, (int2*)nullptr, (int*)nullptr,
                  C.flag);
        YK_LAUNCH(k_scan_offsets, 1, 1024, 0, st, (int)g->n, counts, C.off);
        int total = 0;
        YK_TRY_CUDA(cudaMemcpyAsync(&total, C.off + g->n, sizeof(int), cudaMemcpyDeviceToHost, st));
        YK_TRY_CUDA(cudaMemsetAsync(C.flag + 1, 0, sizeof(int), st));   // node counter
        YK_TRY_CUDA(cudaStreamSynchronize(st));
        if (total > 0) {
            YK_TRY(grow_int((void**)&C.ent, &C.cap, total, sizeof(int2), st));
            YK_LAUNCH(k_contact_entries<true>, ceil_div(g->n, 256), 256, 0, st, G, C.partners,
                      C.npartners, (int*)nullptr, C.off, C.ent, C.tgt, C.flag);
            YK_TRY_CUDA(cudaMemcpyAsync(hf, C.flag, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
            YK_TRY_CUDA(cudaStreamSynchronize(st));
            C.ntgt = hf[1];
        }
    }
    YK_TRY_CUDA(cudaGetLastError());
    C.valid = true;
    return YK_OK;
}

int contact_apply(yk_geom* g, const double* sigma, double* y, bool grad) {
    Contact& C = g->contact;
    if (!C.valid) YK_TRY(contact_build(g));
    if (C.ntgt == 0) return YK_OK;
    cudaStream_t st = g->ctx->stream;
    GeomView G = g->view();
    const int os = g->prm.oversample;
    if (grad)
        YK_LAUNCH(k_contact_apply<true>, ceil_div((int64_t)C.ntgt * 32, 128), 128, 0, st, G,
                  g->d_particles, sigma, C.off, C.ent, C.tgt, C.ntgt, os, g->d_fine_x,
                  g->d_fine_w, g->d_interp, y);
    else
        YK_LAUNCH(k_contact_apply<false>, ceil_div((int64_t)C.ntgt * 32, 128), 128, 0, st, G,
                  g->d_particles, sigma, C.off, C.ent, C.tgt, C.ntgt, os, g->d_fine_x,
                  g->d_fine_w, g->d_interp, y);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

int contact_targets(yk_geom* g, int* ntgt) {
    Contact& C = g->contact;
    if (!C.valid) YK_TRY(contact_build(g));
    *ntgt = C.ntgt;
    return YK_OK;
}

void contact_free(yk_geom* g) {
    Contact& C = g->contact;
    cudaStream_t st = g->ctx->stream;
    void* bufs[] = {C.partners, C.npartners, C.off, C.tgt, C.flag, C.ent};
    for (void* b : bufs) dev_free(b, st);
    C = Contact{};
}

}  // namespace yk
