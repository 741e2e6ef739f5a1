// Particle dynamics with constant drag coefficients (Algorithm 1 with the
// update of Eq. euler) and the excluded-volume repulsion of Eq. repul.
//
// Repulsion (Section S1): an ellipse (A > B) is three circles of radius B at
// a_i + k h d_i, h = A - B, k in {-1, 0, +1}, d_i = (cos theta_i, sin theta_i);
// a disk is one circle of its radius. Every pair of circles of different
// particles repels by Eq. repul,
//   f = c q / (|c_i - c_j| - (b_i + b_j))^{q+1} (c_i - c_j)/|c_i - c_j|,
// with c = c0 / (n_i n_j) (n = circles per particle), so that two circles
// recover Eq. repul exactly; the torque about a_i is the lever arm k h d_i
// crossed with f, and the potential c / (|c_i - c_j| - (b_i + b_j))^q is
// shared half and half.
//
// Step: label, GMRES (warm-started from the previous density), hydrophobic
// force and torque (Eqs. force_torque, stress, scalar-torque), repulsion,
// a += dt (F + F_rep) / xi_x, theta += dt (tau + tau_rep) / xi_theta, then
// the boundary is re-discretised at the new positions.
#include <math.h>

#include <cstring>
#include <vector>

#include "yk_internal.cuh"

namespace yk {

struct Circles {
    int n;
    double cx[3], cy[3], ax[3], ay[3];   // centres and lever arms
    double r;
};

__device__ __forceinline__ Circles circles_of(const yk_particle& P) {
    Circles c;
    if (P.shape == YK_SHAPE_DISK || P.A == P.B) {
        c.n = 1;
        c.cx[0] = P.cx;
        c.cy[0] = P.cy;
        c.ax[0] = c.ay[0] = 0.0;
        c.r = P.A;
        return c;
    }
    double s, co;
    sincos(P.phi, &s, &co);
    const double h = P.A - P.B;
    c.n = 3;
    for (int k = 0; k < 3; ++k) {
        c.ax[k] = (k - 1) * h * co;
        c.ay[k] = (k - 1) * h * s;
        c.cx[k] = P.cx + c.ax[k];
        c.cy[k] = P.cy + c.ay[k];
    }
    c.r = P.B;
    return c;
}

__device__ __forceinline__ double ipow(double x, int q) {
    double r = 1.0;
    for (int k = 0; k < q; ++k) r *= x;
    return r;
}

// F[2i], tau[i], phi[i] for every particle i (one thread each, all j).
// *bad is set when two circles overlap (no finite repulsion).
__global__ void k_repulsion(int np, const yk_particle* __restrict__ parts, double c0, int q,
                            double* __restrict__ F, double* __restrict__ tau,
                            double* __restrict__ phi, int* __restrict__ bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const Circles ci = circles_of(parts[i]);
    double fx = 0.0, fy = 0.0, tq = 0.0, en = 0.0;
    for (int j = 0; j < np; ++j) {
        if (j == i) continue;
        const Circles cj = circles_of(parts[j]);
        const double c = c0 / (double)(ci.n * cj.n);
        for (int k = 0; k < ci.n; ++k)
            for (int l = 0; l < cj.n; ++l) {
                const double dx = ci.cx[k] - cj.cx[l], dy = ci.cy[k] - cj.cy[l];
                const double dist = sqrt(dx * dx + dy * dy);
                const double s = dist - (ci.r + cj.r);
                if (!(s > 0.0)) {
                    atomicExch(bad, 1);
                    continue;
                }
                const double sq = ipow(s, q);
                const double mag = c * q / (sq * s) / dist;
                const double gx = mag * dx, gy = mag * dy;
                fx += gx;
                fy += gy;
                tq += ci.ax[k] * gy - ci.ay[k] * gx;
                en += 0.5 * c / sq;
            }
    }
    F[2 * i] = fx;
    F[2 * i + 1] = fy;
    tau[i] = tq;
    phi[i] = en;
}

// Eq. euler with the total force and torque.
__global__ void k_euler(int np, yk_particle* __restrict__ parts, const double* __restrict__ F,
                        const double* __restrict__ tau, const double* __restrict__ Fr,
                        const double* __restrict__ taur, double dt, double xi_x,
                        double xi_theta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    yk_particle& P = parts[i];
    P.cx += dt * (F[2 * i] + Fr[2 * i]) / xi_x;
    P.cy += dt * (F[2 * i + 1] + Fr[2 * i + 1]) / xi_x;
    P.phi += dt * (tau[i] + taur[i]) / xi_theta;
}

// F += Fr, tau += taur (the loads of Eq. mobility_bc)
__global__ void k_add_loads(int np, double* __restrict__ F, double* __restrict__ tau,
                            const double* __restrict__ Fr, const double* __restrict__ taur) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    F[2 * i] += Fr[2 * i];
    F[2 * i + 1] += Fr[2 * i + 1];
    tau[i] += taur[i];
}

// Eq. mob_vec by forward Euler: a += dt v, theta += dt omega.
__global__ void k_move(int np, yk_particle* __restrict__ parts, const double* __restrict__ v,
                       const double* __restrict__ om, double dt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    parts[i].cx += dt * v[2 * i];
    parts[i].cy += dt * v[2 * i + 1];
    parts[i].phi += dt * om[i];
}

// Device copy of the particles and the step buffers, allocated on first use.
static int dyn_buffers(yk_geom* g) {
    Dynamics& D = g->dyn;
    if (D.parts) return YK_OK;
    cudaStream_t st = g->ctx->stream;
    YK_TRY(dev_alloc((void**)&D.parts, sizeof(yk_particle) * g->np, st));
    YK_TRY(dev_alloc((void**)&D.sigma, sizeof(double) * g->n, st));
    YK_TRY(dev_alloc((void**)&D.f, sizeof(double) * g->n, st));
    YK_TRY(dev_alloc((void**)&D.un, sizeof(double) * g->n, st));
    YK_TRY(dev_alloc((void**)&D.work, sizeof(double) * (9 * (size_t)g->np + 8), st));
    YK_TRY(dev_alloc((void**)&D.bad, sizeof(int), st));
    return YK_OK;
}

void dyn_free(yk_geom* g) {
    Dynamics& D = g->dyn;
    cudaStream_t st = g->ctx->stream;
    void* bufs[] = {D.parts, D.sigma, D.f, D.un, D.work, D.bad};
    for (void* b : bufs) dev_free(b, st);
    D = Dynamics{};
}

int repulsion(yk_geom* g, const yk_particle* d_parts, double c0, int q, double* F, double* tau,
              double* phi) {
    YK_TRY(dyn_buffers(g));
    cudaStream_t st = g->ctx->stream;
    YK_TRY_CUDA(cudaMemsetAsync(g->dyn.bad, 0, sizeof(int), st));
    YK_LAUNCH(k_repulsion, ceil_div(g->np, 128), 128, 0, st, g->np, d_parts, c0, q, F, tau, phi,
              g->dyn.bad);
    int bad = 0;
    YK_TRY_CUDA(cudaMemcpyAsync(&bad, g->dyn.bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    return bad ? YK_ERR_BAD_GEOMETRY : YK_OK;
}

int repulsion_host(yk_geom* g, double c0, int q, double* F, double* tau, double* phi) {
    YK_TRY(dyn_buffers(g));
    cudaStream_t st = g->ctx->stream;
    YK_TRY_CUDA(cudaMemcpyAsync(g->dyn.parts, g->parts.data(), sizeof(yk_particle) * g->np,
                                cudaMemcpyHostToDevice, st));
    return repulsion(g, g->dyn.parts, c0, q, F, tau, phi);
}

int step(yk_geom* g, const yk_dynamics& d, yk_solve_info* info, double* energy_out) {
    YK_TRY(dyn_buffers(g));
    Dynamics& D = g->dyn;
    cudaStream_t st = g->ctx->stream;
    const int np = g->np;
    double* F = D.work;
    double* tau = F + 2 * np;
    double* Fr = tau + np;
    double* taur = Fr + 2 * np;
    double* phi = taur + np;
    double* phir = phi + np;
    double* tot = phir + np;   // 2 doubles
    YK_TRY(launch_label(g, d.label_kind, d.label_param, D.f));
    const bool warm = d.warm_start && D.have_sigma;
    yk_solve_info inf{};
    const int rc = solve(g, D.f, D.sigma, warm ? D.sigma : nullptr, &inf);
    if (info) *info = inf;
    YK_TRY(rc);   // a solve that did not converge moves nothing
    D.have_sigma = true;
    YK_TRY(normal_derivative(g, D.sigma, D.un,
                             g->prm.precision == YK_FP64 ? Prec::F64 : Prec::SPLIT));
    YK_TRY(forces_torques(g, D.sigma, D.f, D.un, F, tau, nullptr));
    YK_TRY_CUDA(cudaMemcpyAsync(D.parts, g->parts.data(), sizeof(yk_particle) * np,
                                cudaMemcpyHostToDevice, st));
    YK_TRY(repulsion(g, D.parts, d.c0, d.q, Fr, taur, phir));
    if (energy_out) {
        // Phi of Eq. main plus the repulsion potential, at the configuration
        // the step starts from
        YK_TRY(energy(g, D.f, D.un, phi, tot));
        std::vector<double> hp(np);
        double e = 0.0;
        YK_TRY_CUDA(cudaMemcpyAsync(&e, tot, sizeof(double), cudaMemcpyDeviceToHost, st));
        YK_TRY_CUDA(cudaMemcpyAsync(hp.data(), phir, sizeof(double) * np, cudaMemcpyDeviceToHost,
                                    st));
        YK_TRY_CUDA(cudaStreamSynchronize(st));
        for (double v : hp) e += v;
        *energy_out = e;
    }
    if (d.mobility) {
        // Eq. mob_vec: the velocities of the Stokes mobility problem under the
        // total loads (Eq. mobility_bc), then forward Euler
        double* V = phi;            // 2 np (phi, phir are free after the energy)
        double* Om = tot + 2;       // np
        YK_LAUNCH(k_add_loads, ceil_div(np, 128), 128, 0, st, np, F, tau, Fr, taur);
        const int rc = mobility(g, F, tau, V, Om, nullptr, nullptr);
        YK_TRY(rc);
        YK_LAUNCH(k_move, ceil_div(np, 128), 128, 0, st, np, D.parts, V, Om, d.dt);
    } else {
        YK_LAUNCH(k_euler, ceil_div(np, 128), 128, 0, st, np, D.parts, F, tau, Fr, taur, d.dt,
                  d.xi_x, d.xi_theta);
    }
    std::vector<yk_particle> moved(np);
    YK_TRY_CUDA(cudaMemcpyAsync(moved.data(), D.parts, sizeof(yk_particle) * np,
                                cudaMemcpyDeviceToHost, st));
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < np; ++i) {
        g->parts[i].cx = moved[i].cx;
        g->parts[i].cy = moved[i].cy;
        g->parts[i].phi = moved[i].phi;
    }
    return update_nodes(g);
}

}  // namespace yk
