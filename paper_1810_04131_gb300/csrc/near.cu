// The potential u = D[sigma](t) (Eq. intrep) at targets anywhere in the
// water, including targets arbitrarily close to a boundary, by QBX for the
// panels next to the target (Section 5; the paper's Table 1 samples such
// targets on a 200 x 200 grid).
//
// For each particle P and target t:
//   * t inside P: the result is NaN;
//   * p = the boundary point of P closest to t (Newton's method on the curve
//     parameter in P's body frame, from the nearest node), d = |t - p|;
//   * d >= near_factor x (largest panel arclength of P's shape): plain
//     quadrature over P's nodes;
//   * otherwise the panels next to p (p's panel +- near_width) are taken out
//     of the plain quadrature and evaluated
//       - for d <= 2r (r = r_factor x p's panel arclength) by the local
//         expansion u = sum_{|n|<=p} alpha_n I_n(|t-c|/rho) e^{in theta} about
//         the target's own centre c = p + r nu(p), on the normal through p (so
//         |t - c| = |d - r| <= r), with
//         alpha_n = (1/2pi) int sigma nu . grad_y[K_n(|y-c|/rho) e^{-in phi_y}] ds
//         from the oversampled panels (sigma interpolated), as for the
//         on-surface targets of the QBX rows;
//       - else by quadrature on the oversampled nodes.
// Everything next to P is evaluated in P's body frame (the field depends on
// relative positions only).
#include <math.h>

#include <algorithm>
#include <vector>

#include "bessel.cuh"
#include "yk_internal.cuh"

namespace yk {

constexpr int NEAR_SLOTS = 4;       // near particles per target
constexpr double NEAR_FACTOR = 1.0; // near zone: d < NEAR_FACTOR x largest panel arclength
constexpr int NEAR_TPB = 128;
constexpr int NEAR_STILE = 256;

struct NearEntry {
    int P;          // particle (-1: empty slot)
    int kp;         // panel holding the closest point
    int mode;       // 1: QBX about (cx, cy); 2: oversampled quadrature
    int pad_;
    double cx, cy;  // expansion centre, P's body frame
    double tx, ty;  // target, P's body frame
};

__device__ __forceinline__ void body_point(double A, double B, double t, double& x, double& y,
                                           double& dx, double& dy) {
    double s, c;
    sincos(t, &s, &c);
    x = A * c;
    y = B * s;
    dx = -A * s;
    dy = B * c;
}

// Arclength of panel k of the shape (A, B): the sum of its node weights.
__device__ double panel_length(double A, double B, int k, int npan, int ngl,
                               const double* glx, const double* glw) {
    const double dt = 2.0 * PI / npan;
    double h = 0.0;
    for (int m = 0; m < ngl; ++m) {
        double x, y, dx, dy;
        body_point(A, B, k * dt + 0.5 * dt * (glx[m] + 1.0), x, y, dx, dy);
        h += glw[m] * 0.5 * dt * sqrt(dx * dx + dy * dy);
    }
    return h;
}

// Largest panel arclength of each shape (one block per shape).
__global__ void k_shape_hmax(int npan, int ngl, const double2* __restrict__ shape_ab,
                             const double* __restrict__ glx, const double* __restrict__ glw,
                             double* __restrict__ hmax) {
    __shared__ double red[NEAR_TPB];
    const int s = blockIdx.x;
    double h = 0.0;
    for (int k = threadIdx.x; k < npan; k += blockDim.x)
        h = fmax(h, panel_length(shape_ab[s].x, shape_ab[s].y, k, npan, ngl, glx, glw));
    red[threadIdx.x] = h;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) hmax[s] = red[0];
}

// Closest boundary point of the ellipse (A cos s, B sin s) to (tx, ty), body
// frame: Newton's method on (x(s) - t) . x'(s) = 0 from s0.
__device__ double closest_param(double A, double B, double tx, double ty, double s0) {
    double s = s0;
    for (int it = 0; it < 50; ++it) {
        double x, y, dx, dy;
        body_point(A, B, s, x, y, dx, dy);
        const double ex = x - tx, ey = y - ty;
        const double f = ex * dx + ey * dy;
        const double fp = dx * dx + dy * dy - (ex * x + ey * y);   // x'' = -x
        const double step = f / fp;
        s -= step;
        if (fabs(step) < 1e-15) break;
    }
    return s;
}

// Near entries of every target (one thread each); inside[t] = 1 for a target
// inside a particle; *overflow = 1 when a target is near more than
// NEAR_SLOTS particles.
__global__ void k_near_find(GeomView G, const yk_particle* __restrict__ parts,
                            const double* __restrict__ hmax, const double* __restrict__ glx,
                            const double* __restrict__ glw, double r_factor,
                            const double* __restrict__ tgt, int64_t nt,
                            NearEntry* __restrict__ ent, int* __restrict__ inside,
                            int* __restrict__ overflow) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double tx = tgt[2 * t], ty = tgt[2 * t + 1];
    const double dtp = 2.0 * PI / G.npan;
    int ns = 0, in = 0;
    for (int P = 0; P < G.np && !in; ++P) {
        const yk_particle pr = parts[P];
        const double hm = hmax[G.shape_of[P]];
        const double rx = tx - pr.cx, ry = ty - pr.cy;
        if (sqrt(rx * rx + ry * ry) >= fmax(pr.A, pr.B) + (NEAR_FACTOR + 1.0) * hm) continue;
        double sp, cp;
        sincos(pr.phi, &sp, &cp);
        const double bx = cp * rx + sp * ry, by = -sp * rx + cp * ry;   // body frame
        if ((bx / pr.A) * (bx / pr.A) + (by / pr.B) * (by / pr.B) < 1.0) {
            in = 1;
            break;
        }
        const int64_t base = (int64_t)P * G.npp;
        double dmin = INFINITY;
        int bmin = 0;
        for (int l = 0; l < G.npp; ++l) {
            const double ex = G.x[base + l] - tx, ey = G.y[base + l] - ty;
            const double d2 = ex * ex + ey * ey;
            if (d2 < dmin) dmin = d2, bmin = l;
        }
        if (sqrt(dmin) >= (NEAR_FACTOR + 1.0) * hm) continue;
        const double s0 = (bmin / G.ngl) * dtp + 0.5 * dtp * (glx[bmin % G.ngl] + 1.0);
        double s = fmod(closest_param(pr.A, pr.B, bx, by, s0), 2.0 * PI);
        if (s < 0.0) s += 2.0 * PI;
        double px, py, dx, dy;
        body_point(pr.A, pr.B, s, px, py, dx, dy);
        const double d = sqrt((bx - px) * (bx - px) + (by - py) * (by - py));
        if (d >= NEAR_FACTOR * hm) continue;
        const int kp = min((int)(s / dtp), G.npan - 1);
        const double r = r_factor * panel_length(pr.A, pr.B, kp, G.npan, G.ngl, glx, glw);
        const double spd = sqrt(dx * dx + dy * dy);
        if (ns == NEAR_SLOTS) {
            atomicExch(overflow, 1);
            break;
        }
        NearEntry e;
        e.P = P;
        e.kp = kp;
        e.mode = (d <= 2.0 * r) ? 1 : 2;
        e.pad_ = 0;
        e.cx = px + r * dy / spd;          // nu = (dy, -dx) / |x'|, out of the particle
        e.cy = py - r * dx / spd;
        e.tx = bx;
        e.ty = by;
        ent[t * NEAR_SLOTS + ns++] = e;
    }
    for (int k = ns; k < NEAR_SLOTS; ++k) ent[t * NEAR_SLOTS + k].P = -1;
    inside[t] = in;
}

__device__ __forceinline__ bool near_panel(int kp, int pq, int npan, int w) {
    if (2 * w + 1 >= npan) return true;
    int d = ((pq - kp) % npan + npan) % npan;
    return d <= w || npan - d <= w;
}

// Plain quadrature of the double layer at the targets over a chunk of source
// particles (blockIdx.y), leaving out each target's near panels.
__global__ void __launch_bounds__(NEAR_TPB) k_near_plain(GeomView G,
                                                         const double* __restrict__ sigma,
                                                         const double* __restrict__ tgt,
                                                         int64_t nt, int ppc,
                                                         const NearEntry* __restrict__ ent,
                                                         double* __restrict__ partial) {
    __shared__ d4 src[NEAR_STILE];
    const int64_t i = blockIdx.x * (int64_t)NEAR_TPB + threadIdx.x;
    const bool active = i < nt;
    const double tx = active ? tgt[2 * i] : 0.0, ty = active ? tgt[2 * i + 1] : 0.0;
    int eP[NEAR_SLOTS], eK[NEAR_SLOTS];
#pragma unroll
    for (int k = 0; k < NEAR_SLOTS; ++k) {
        eP[k] = active ? ent[i * NEAR_SLOTS + k].P : -1;
        eK[k] = active ? ent[i * NEAR_SLOTS + k].kp : 0;
    }
    const double rho = G.rho, kappa = 1.0 / rho, two_rho = 2.0 * rho;
    const int s0 = blockIdx.y * ppc;
    const int s1 = min(G.np, s0 + ppc);
    double acc = 0.0;
    for (int s = s0; s < s1; ++s) {
        int kp = -1;
#pragma unroll
        for (int k = 0; k < NEAR_SLOTS; ++k)
            if (eP[k] == s) kp = eK[k];
        const int64_t base = (int64_t)s * G.npp;
        for (int jb = 0; jb < G.npp; jb += NEAR_STILE) {
            const int cnt = min(NEAR_STILE, G.npp - jb);
            __syncthreads();
            for (int q = threadIdx.x; q < cnt; q += NEAR_TPB) {
                const int64_t j = base + jb + q;
                const double ws = G.w[j] * sigma[j];
                src[q] = make_d4(G.x[j], G.y[j], ws * G.nx[j], ws * G.ny[j]);
            }
            __syncthreads();
            if (!active) continue;
            for (int q = 0; q < cnt; ++q) {
                if (kp >= 0 && near_panel(kp, (jb + q) / G.ngl, G.npan, G.near_w)) continue;
                const d4 S = src[q];
                const double dx = tx - S.x, dy = ty - S.y;
                const double r2 = fma(dx, dx, dy * dy);
                const double ri = rsqrt(r2);
                const double z = r2 * ri * kappa;
                double k1v;
                if (z <= 2.0) k1v = k1_series(z);
                else k1v = exp(-z) * p1_large(two_rho * ri) * rsqrt(z);
                acc = fma(k1v * ri, fma(dx, S.z, dy * S.w), acc);
            }
        }
    }
    if (active) partial[blockIdx.y * nt + i] = acc / (2.0 * PI * rho);
}

// u = sum of the chunk partials (NaN for targets inside a particle).
__global__ void k_near_sum(int64_t nt, int nchunk, const double* __restrict__ partial,
                           const int* __restrict__ inside, double* __restrict__ u) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nt) return;
    double acc = 0.0;
    for (int c = 0; c < nchunk; ++c) acc += partial[c * nt + i];
    u[i] = inside[i] ? nan("") : acc;
}

// The near panels of slot `slot` of every target (one warp per target),
// added to u: the QBX expansion about the entry's centre (mode 1) or
// quadrature on the oversampled nodes (mode 2), all in P's body frame.
__global__ void __launch_bounds__(NEAR_TPB) k_near_corr(GeomView G,
                                                        const double2* __restrict__ shape_ab,
                                                        const double* __restrict__ sigma,
                                                        const NearEntry* __restrict__ ent,
                                                        int slot, int64_t nt, int os, int order,
                                                        const double* __restrict__ fine_x,
                                                        const double* __restrict__ fine_w,
                                                        const double* __restrict__ interp,
                                                        const int* __restrict__ inside,
                                                        double* __restrict__ u) {
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= nt) return;
    const NearEntry e = ent[t * NEAR_SLOTS + slot];
    if (e.P < 0 || inside[t]) return;                   // warp-uniform
    const double2 ab = shape_ab[G.shape_of[e.P]];
    const double rho = G.rho;
    const double dt = 2.0 * PI / G.npan;
    const int nfp = os * G.ngl;
    const int all = (2 * G.near_w + 1 >= G.npan);
    const int nf = G.n_near * nfp;
    const int64_t base = (int64_t)e.P * G.npp;
    double ar[MAX_ORDER + 1], ai[MAX_ORDER + 1];
    for (int n = 0; n <= order; ++n) ar[n] = ai[n] = 0.0;
    double plain = 0.0;
    for (int f = lane; f < nf; f += 32) {
        const int q = f / nfp, m = f % nfp;
        const int pk = all ? q : ((e.kp - G.near_w + q) % G.npan + G.npan) % G.npan;
        double yx, yy, dx, dy;
        body_point(ab.x, ab.y, pk * dt + 0.5 * dt * (fine_x[m] + 1.0), yx, yy, dx, dy);
        const double spd = sqrt(dx * dx + dy * dy);
        const double nux = dy / spd, nuy = -dx / spd;
        const double wf = 0.5 * dt * fine_w[m] * spd;
        double sf = 0.0;                                   // sigma interpolated to the fine node
        for (int j = 0; j < G.ngl; ++j)
            sf = fma(interp[m * G.ngl + j], sigma[base + (int64_t)pk * G.ngl + j], sf);
        const double ws = wf * sf;
        if (e.mode == 2) {
            const double ex = e.tx - yx, ey = e.ty - yy;
            const double r = sqrt(ex * ex + ey * ey);
            plain += k1(r / rho) * (ex * nux + ey * nuy) / r * ws;
            continue;
        }
        const double ex = yx - e.cx, ey = yy - e.cy;
        const double sd = sqrt(ex * ex + ey * ey);
        const double esx = ex / sd, esy = ey / sd;
        const double a_s = nux * esx + nuy * esy;          // nu . e_s
        const double a_p = -nux * esy + nuy * esx;         // nu . e_phi
        const double z = sd / rho;
        double Kn[MAX_ORDER + 2];
        k01(z, Kn[0], Kn[1]);
        for (int n = 1; n <= order; ++n) Kn[n + 1] = Kn[n - 1] + (2.0 * n / z) * Kn[n];
        double cn = 1.0, sn = 0.0;                         // (cos, sin)(n phi)
        for (int n = 0; n <= order; ++n) {
            const double kp = (n == 0) ? -Kn[1] : -0.5 * (Kn[n - 1] + Kn[n + 1]);
            const double br = a_s * kp / rho, bi = -n * a_p * Kn[n] / sd;
            // (br + i bi) e^{-i n phi}
            ar[n] = fma(ws, br * cn + bi * sn, ar[n]);
            ai[n] = fma(ws, bi * cn - br * sn, ai[n]);
            const double c2 = cn * esx - sn * esy;
            sn = sn * esx + cn * esy;
            cn = c2;
        }
    }
    double val;
    if (e.mode == 2) {
        for (int o = 16; o > 0; o >>= 1) plain += __shfl_xor_sync(0xffffffffu, plain, o);
        val = plain / (2.0 * PI * rho);
    } else {
        for (int n = 0; n <= order; ++n)
            for (int o = 16; o > 0; o >>= 1) {
                ar[n] += __shfl_xor_sync(0xffffffffu, ar[n], o);
                ai[n] += __shfl_xor_sync(0xffffffffu, ai[n], o);
            }
        const double vx = e.tx - e.cx, vy = e.ty - e.cy;
        const double rr = sqrt(vx * vx + vy * vy);
        const double x = rr / rho;
        double I[MAX_ORDER + 2];
        if (x < 1e-6) {                                   // I_n(x) = (x/2)^n / n! to 1e-13
            double v = 1.0;
            for (int n = 0; n <= order; ++n) {
                I[n] = v;
                v *= 0.5 * x / (n + 1);
            }
        } else {
            bessel_i_down(order + 1, x, I);
        }
        const double cth = rr > 0.0 ? vx / rr : 1.0, sth = rr > 0.0 ? vy / rr : 0.0;
        double cn = 1.0, sn = 0.0, acc = 0.0;
        for (int n = 0; n <= order; ++n) {
            acc += (n == 0 ? 1.0 : 2.0) * I[n] * (ar[n] * cn - ai[n] * sn);   // Re[alpha_n e^{in theta}]
            const double c2 = cn * cth - sn * sth;
            sn = sn * cth + cn * sth;
            cn = c2;
        }
        val = acc / (2.0 * PI);
    }
    if (lane == 0) u[t] += val;
}

int potential_near(yk_geom* g, const double* sigma, const double* targets, int64_t nt,
                   double* u) {
    if (nt <= 0) return YK_OK;
    cudaStream_t st = g->ctx->stream;
    GeomView G = g->view();
    const int np = g->np;
    yk_particle* d_parts = nullptr;
    double* hmax = nullptr;
    NearEntry* ent = nullptr;
    int* inside = nullptr;
    double* part = nullptr;
    const int nct = ceil_div(nt, NEAR_TPB);
    int nchunk = std::max(1, std::min(np, ceil_div(4 * 152, nct)));
    const int ppc = ceil_div(np, nchunk);
    nchunk = ceil_div(np, ppc);
    int rc = YK_OK;
    auto al = [&](void** p, size_t b) {
        if (rc == YK_OK && cudaMallocAsync(p, b, st) != cudaSuccess) rc = YK_ERR_NO_MEMORY;
    };
    al((void**)&d_parts, sizeof(yk_particle) * np);
    al((void**)&hmax, sizeof(double) * g->nshape);
    al((void**)&ent, sizeof(NearEntry) * NEAR_SLOTS * (size_t)nt);
    al((void**)&inside, sizeof(int) * ((size_t)nt + 1));
    al((void**)&part, sizeof(double) * nchunk * (size_t)nt);
    int overflow = 0;
    if (rc == YK_OK) {
        int* d_over = inside + nt;
        cudaMemcpyAsync(d_parts, g->parts.data(), sizeof(yk_particle) * np,
                        cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(d_over, 0, sizeof(int), st);
        YK_LAUNCH(k_shape_hmax, g->nshape, NEAR_TPB, 0, st, g->npan, g->ngl, g->d_shape_ab,
                  g->d_glx, g->d_glw, hmax);
        YK_LAUNCH(k_near_find, ceil_div(nt, 128), 128, 0, st, G, d_parts, hmax, g->d_glx,
                  g->d_glw, g->prm.qbx_r_factor, targets, nt, ent, inside, d_over);
        YK_LAUNCH(k_near_plain, dim3(nct, nchunk), NEAR_TPB, 0, st, G, sigma, targets, nt, ppc,
                  ent, part);
        YK_LAUNCH(k_near_sum, ceil_div(nt, 256), 256, 0, st, nt, nchunk, part, inside, u);
        for (int k = 0; k < NEAR_SLOTS; ++k)
            YK_LAUNCH(k_near_corr, ceil_div(nt * 32, NEAR_TPB), NEAR_TPB, 0, st, G, g->d_shape_ab,
                      sigma, ent, k, nt, g->prm.oversample, g->prm.qbx_order, g->d_fine_x,
                      g->d_fine_w, g->d_interp, inside, u);
        if (cudaGetLastError() != cudaSuccess) rc = YK_ERR_CUDA;
        if (rc == YK_OK &&
            (cudaMemcpyAsync(&overflow, d_over, sizeof(int), cudaMemcpyDeviceToHost, st) !=
                 cudaSuccess ||
             cudaStreamSynchronize(st) != cudaSuccess))
            rc = YK_ERR_CUDA;
    }
    void* bufs[] = {d_parts, hmax, ent, inside, part};
    for (void* b : bufs)
        if (b) cudaFreeAsync(b, st);
    if (rc == YK_OK && overflow) rc = YK_ERR_TOO_LARGE;
    return rc;
}

}  // namespace yk
