// Hydrophobic force and torque on each particle (Eqs. force_torque, stress,
// scalar-torque). On the boundary grad u = u_nu nu + u_tau tau, with u_nu
// from the exterior normal derivative of D[sigma] and u_tau = df/ds
// (u = f on the boundary) by per-panel Lagrange differentiation in the
// curve parameter divided by the speed. The stress applied to the particle
// normal nu is
//   T.nu = gamma [f^2/rho + rho u_tau^2 - rho u_nu^2] nu - 2 gamma rho u_nu u_tau tau,
//   F_i = sum_nodes w T.nu,  tau0_i = sum_nodes w (x cross T.nu),
//   tau_i = tau0_i - a_i cross F_i   (2-D cross a x b = a_x b_y - a_y b_x).
//
// Energy (Eq. main): Phi = gamma min I[u], I[u] = int_Omega rho |grad u|^2 +
// u^2/rho dx. Green's first identity on the water domain (outward normal
// -nu) with Delta u = u/rho^2 (Eq. SL) and u -> 0 at infinity leaves the
// boundary form Phi = -gamma rho sum_i int_{Sigma_i} f u_nu ds, summed per
// particle here from the same u_nu as the forces.
#include "yk_internal.cuh"

namespace yk {

constexpr int FT_TPB = 256;

__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
    __shared__ double red[3][FT_TPB];
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    red[2][threadIdx.x] = c;
    __syncthreads();
    for (int o = FT_TPB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            red[0][threadIdx.x] += red[0][threadIdx.x + o];
            red[1][threadIdx.x] += red[1][threadIdx.x + o];
            red[2][threadIdx.x] += red[2][threadIdx.x + o];
        }
        __syncthreads();
    }
    a = red[0][0];
    b = red[1][0];
    c = red[2][0];
}

__global__ void __launch_bounds__(FT_TPB) k_forces(GeomView G, const double* __restrict__ diff,
                                                   const double* __restrict__ f,
                                                   const double* __restrict__ un, double gamma,
                                                   double* __restrict__ F, double* __restrict__ tau,
                                                   double* __restrict__ tau0) {
    const int p = blockIdx.x;
    const int64_t base = (int64_t)p * G.npp;
    const double rho = G.rho;
    const double dscale = 2.0 / (2.0 * PI / G.npan);   // d/dt = (2/dt) d/dxi
    double fx = 0.0, fy = 0.0, tq = 0.0;
    for (int li = threadIdx.x; li < G.npp; li += FT_TPB) {
        const int k = li / G.ngl, j = li % G.ngl;
        const int64_t i = base + li;
        const double* fp = f + base + (int64_t)k * G.ngl;
        double dfd = 0.0;
        for (int m = 0; m < G.ngl; ++m) dfd = fma(diff[j * G.ngl + m], fp[m], dfd);
        const double ut = dfd * dscale / G.speed[i];
        const double u = f[i], unn = un[i];
        const double nx = G.nx[i], ny = G.ny[i];
        const double tx = -ny, ty = nx;
        const double sn = gamma * (u * u / rho + rho * ut * ut - rho * unn * unn);
        const double st = -2.0 * gamma * rho * unn * ut;
        const double w = G.w[i];
        const double Tx = w * (sn * nx + st * tx);
        const double Ty = w * (sn * ny + st * ty);
        fx += Tx;
        fy += Ty;
        tq += G.x[i] * Ty - G.y[i] * Tx;
    }
    block_sum3(fx, fy, tq);
    if (threadIdx.x == 0) {
        const yk::d4 a = G.part[p];
        F[2 * p] = fx;
        F[2 * p + 1] = fy;
        tau0[p] = tq;
        tau[p] = tq - (a.x * fy - a.y * fx);
    }
}

// net[0..3) = sum F_x, sum F_y, sum tau0 (Eq. net)
__global__ void k_net(int np, const double* __restrict__ F, const double* __restrict__ tau0,
                      double* __restrict__ net) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int p = threadIdx.x; p < np; p += FT_TPB) {
        a += F[2 * p];
        b += F[2 * p + 1];
        c += tau0[p];
    }
    block_sum3(a, b, c);
    if (threadIdx.x == 0) {
        net[0] = a;
        net[1] = b;
        net[2] = c;
    }
}

// phi[p] = -gamma rho sum over particle p's nodes of w f u_nu; total[0] = sum_p phi[p]
__global__ void __launch_bounds__(FT_TPB) k_energy(GeomView G, const double* __restrict__ f,
                                                   const double* __restrict__ un, double gamma,
                                                   double* __restrict__ phi) {
    const int p = blockIdx.x;
    const int64_t base = (int64_t)p * G.npp;
    double e = 0.0, z1 = 0.0, z2 = 0.0;
    for (int li = threadIdx.x; li < G.npp; li += FT_TPB) {
        const int64_t i = base + li;
        e = fma(G.w[i] * f[i], un[i], e);
    }
    block_sum3(e, z1, z2);
    if (threadIdx.x == 0) phi[p] = -gamma * G.rho * e;
}

__global__ void k_energy_total(int np, const double* __restrict__ phi, double* __restrict__ total) {
    double a = 0.0, z1 = 0.0, z2 = 0.0;
    for (int p = threadIdx.x; p < np; p += FT_TPB) a += phi[p];
    block_sum3(a, z1, z2);
    if (threadIdx.x == 0) total[0] = a;
}

int energy(yk_geom* g, const double* f, const double* un, double* phi, double* total) {
    cudaStream_t st = g->ctx->stream;
    YK_LAUNCH(k_energy, g->np, FT_TPB, 0, st, g->view(), f, un, g->prm.gamma, phi);
    if (total) YK_LAUNCH(k_energy_total, 1, FT_TPB, 0, st, g->np, phi, total);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

int forces_torques(yk_geom* g, const double* sigma, const double* f, const double* un,
                   double* F, double* tau, double* net) {
    (void)sigma;
    cudaStream_t st = g->ctx->stream;
    double* tau0 = nullptr;
    YK_TRY_CUDA(cudaMallocAsync((void**)&tau0, sizeof(double) * g->np, st));
    YK_LAUNCH(k_forces, g->np, FT_TPB, 0, st, g->view(), g->d_diff, f, un, g->prm.gamma, F, tau, tau0);
    if (net) YK_LAUNCH(k_net, 1, FT_TPB, 0, st, g->np, F, tau0, net);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(tau0, st);
    YK_TRY_CUDA(e);
    return YK_OK;
}

}  // namespace yk
