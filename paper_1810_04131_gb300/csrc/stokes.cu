// The Stokes mobility step (Section 3: Eqs. stokes, mobility_bc, stokesjump,
// mobilityu, mob_vec; Algorithm 1, the steps that solve for mu and update the
// particle velocities) on the geometry's boundary nodes.
//
// Given forces F_i and torques tau_i (Eq. mobility_bc), the density on dP_i
// is sigma = sigma_inc + mu with
//   sigma_inc = F_i / |dP_i| + tau_i (y - a_i)^perp / J_i,  J_i = int |y - a_i|^2 ds,
// carrying the loads, and mu solving
//   (1/2 I + K* + W) mu = -(1/2 I + K*) sigma_inc,
// where (1/2 I + K*) sigma is the traction of u = S[sigma] (stokeslet single
// layer) on the inside of each boundary (the interior limit of Eq.
// stokesjump, the stresslet T = -(1/pi) r r r / r^4 contracted with the
// target normal) and W projects each boundary's density on its rigid motions
// (1, 0), (0, 1), (y - a_i)^perp. A vanishing interior traction makes u a
// rigid motion on every boundary; v_i and omega_i are the averages of
// Eq. mobilityu. The stokeslet is G = (1/(4 pi mu)) (-log r I + r r^T / r^2)
// (the divergence-free sign of the log).
//
// Layout and kernels:
//   * per particle shape, in the body frame (centre 0, phi = 0), dense
//     2 npp x 2 npp FP64 blocks, column-major: B0 = 1/2 I + K* (own
//     particle, Nystrom with the curvature limit on the diagonal), B = B0 + W
//     (and its FP32 copy for the inner operator), and the single layer S with
//     the log integrated by product integration on the target's panel and its
//     two neighbours (moments of log|xi0 - xi| against the panel's Lagrange
//     basis, by graded Gauss-Legendre quadrature on the device). A particle
//     turned by phi applies R B R^T: its density is turned into the body
//     frame as it is loaded and the result turned back as it is stored;
//   * other particles: dense pair sums, FP64 (x, y, w sigma) records, or FP32
//     offsets from each particle's centre with the centre difference formed
//     in FP64 (inner operator); targets of one particle per block, source
//     particles split over grid.y and added with FP64 atomics;
//   * vectors are node-major (x and y component of node 0, then node 1, ...).
#include <math.h>

#include <algorithm>
#include <vector>

#include "yk_internal.cuh"

namespace yk {

namespace {

constexpr double S_PI = 3.14159265358979323846;
constexpr int QGL = 16;           // graded quadrature rule of the log moments
constexpr int MOMENT_LEVELS = 34; // geometric levels towards a singular point
constexpr int FAR_TPB = 128;
constexpr int FAR_TMAX = 4;       // targets per thread (npp <= FAR_TPB * FAR_TMAX)

__device__ double lagrange(const double* xk, int ngl, int k, double x) {
    double v = 1.0;
    for (int m = 0; m < ngl; ++m)
        if (m != k) v *= (x - xk[m]) / (xk[k] - xk[m]);
    return v;
}

// sum over [a, b] of log|x0 - x| L_k(x) by the QGL-point rule in (qx, qw)
__device__ double log_piece(const double* qx, const double* qw, const double* xk, int ngl, int k,
                            double x0, double a, double b) {
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double s = 0.0;
    for (int m = 0; m < QGL; ++m) {
        const double x = c + h * qx[m];
        s += qw[m] * log(fabs(x0 - x)) * lagrange(xk, ngl, k, x);
    }
    return s * h;
}

// Gauss-Legendre rule of QGL points by Newton's method on P_QGL.
__device__ void gl_rule(double* qx, double* qw) {
    for (int i = threadIdx.x; i < QGL; i += blockDim.x) {
        double x = cos(S_PI * (i + 0.75) / (QGL + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= QGL; ++k) {
                const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = QGL * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        qx[i] = x;
        qw[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

}  // namespace

// M[o][i][k] = int_{-1}^{1} log|xi0 - xi| L_k(xi) dxi at xi0 = xi_i (o = 0),
// xi_i + 2 (o = 1: source panel before the target's), xi_i - 2 (o = 2: after).
// Block (o, i), thread k. Composite Gauss-Legendre on intervals halving
// towards the singular point (inside) or the panel end next to it (outside),
// so that every interval is at least its own length away from it; inside,
// the last 2^-34 of each side is integrated in closed form.
__global__ void k_log_moments(int ngl, const double* __restrict__ glx, double* __restrict__ M) {
    __shared__ double qx[QGL], qw[QGL], xk[64];
    gl_rule(qx, qw);
    for (int m = threadIdx.x; m < ngl; m += blockDim.x) xk[m] = glx[m];
    __syncthreads();
    const int o = blockIdx.x / ngl, i = blockIdx.x % ngl, k = threadIdx.x;
    if (k >= ngl) return;
    const double x0 = xk[i] + (o == 0 ? 0.0 : (o == 1 ? 2.0 : -2.0));
    double s = 0.0;
    if (o == 0) {
        for (int side = 0; side < 2; ++side) {
            const double len = side == 0 ? x0 + 1.0 : 1.0 - x0;
            const double dir = side == 0 ? -1.0 : 1.0;
            double far = len;
            for (int j = 0; j < MOMENT_LEVELS; ++j) {
                const double near = 0.5 * far;
                const double a = x0 + dir * far, b = x0 + dir * near;
                s += log_piece(qx, qw, xk, ngl, k, x0, fmin(a, b), fmax(a, b));
                far = near;
            }
            // the last stretch, of length far < 1e-10 next to x0 = xi_i, where
            // L_k = delta_ik + O(far): int_0^far log u du = far (log far - 1)
            if (k == i) s += far * (log(far) - 1.0);
        }
    } else {
        const double delta = fabs(x0) - 1.0;           // distance to the near panel end
        const double dir = o == 1 ? 1.0 : -1.0;        // the near end is dir * 1
        double h = 1.0;                                 // interval [end - 2h, end - h]
        while (h > delta) {
            const double a = dir * (1.0 - 2.0 * h), b = dir * (1.0 - h);
            s += log_piece(qx, qw, xk, ngl, k, x0, fmin(a, b), fmax(a, b));
            h *= 0.5;
        }
        const double a = dir * (1.0 - 2.0 * h), b = dir * 1.0;
        s += log_piece(qx, qw, xk, ngl, k, x0, fmin(a, b), fmax(a, b));
    }
    M[((int64_t)o * ngl + i) * ngl + k] = s;
}

namespace {

struct BodyNode {
    double x, y, tx, ty, nx, ny, w, spd, kappa;
};

__device__ BodyNode body_node(int li, int ngl, double dt, const double* glx, const double* glw,
                              double A, double B) {
    const int k = li / ngl, a = li % ngl;
    const double t = k * dt + 0.5 * dt * (glx[a] + 1.0);
    double st, ct;
    sincos(t, &st, &ct);
    BodyNode b;
    b.x = A * ct;
    b.y = B * st;
    const double dx = -A * st, dy = B * ct;
    b.spd = sqrt(dx * dx + dy * dy);
    b.tx = dx / b.spd;
    b.ty = dy / b.spd;
    b.nx = b.ty;
    b.ny = -b.tx;
    b.w = glw[a] * 0.5 * dt * b.spd;
    b.kappa = A * B / (b.spd * b.spd * b.spd);
    return b;
}

}  // namespace

// Per shape: perimeter L and J = sum w |x|^2 of the body-frame nodes.
__global__ void k_shape_LJ(int npan, int ngl, const double2* __restrict__ ab,
                           const double* __restrict__ glx, const double* __restrict__ glw,
                           double* __restrict__ LJ) {
    const int s = blockIdx.x;
    const int npp = npan * ngl;
    const double dt = 2.0 * S_PI / npan;
    double l = 0.0, j = 0.0;
    for (int i = threadIdx.x; i < npp; i += blockDim.x) {
        const BodyNode b = body_node(i, ngl, dt, glx, glw, ab[s].x, ab[s].y);
        l += b.w;
        j += b.w * (b.x * b.x + b.y * b.y);
    }
    __shared__ double rl[256], rj[256];
    rl[threadIdx.x] = l;
    rj[threadIdx.x] = j;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            rl[threadIdx.x] += rl[threadIdx.x + o];
            rj[threadIdx.x] += rj[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        LJ[2 * s] = rl[0];
        LJ[2 * s + 1] = rj[0];
    }
}

// The body-frame blocks of one shape: thread (i, j) writes the 2 x 2 entries
// of target node i and source node j of B0 = 1/2 I + K*, B = B0 + W and S.
// Column-major: entry (row 2 i + a, col 2 j + b) at (2 j + b) * 2 npp + 2 i + a.
__global__ void k_stokes_blocks(int npan, int ngl, double visc, const double2* __restrict__ ab,
                                const double* __restrict__ glx, const double* __restrict__ glw,
                                const double* __restrict__ M, const double* __restrict__ LJ,
                                double* __restrict__ B0, double* __restrict__ Bw,
                                double* __restrict__ S) {
    const int s = blockIdx.y;
    const int npp = npan * ngl;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)npp * npp) return;
    const int i = (int)(e % npp), j = (int)(e / npp);
    const double dt = 2.0 * S_PI / npan, half = 0.5 * dt;
    const double A = ab[s].x, Bs = ab[s].y;
    const BodyNode ti = body_node(i, ngl, dt, glx, glw, A, Bs);
    const BodyNode sj = body_node(j, ngl, dt, glx, glw, A, Bs);
    const double L = LJ[2 * s], J = LJ[2 * s + 1];
    double T[2][2], G[2][2];
    const double rx = ti.x - sj.x, ry = ti.y - sj.y;
    const double r2 = rx * rx + ry * ry;
    double rr[2][2];
    if (i == j) {
        const double c = -ti.w * ti.kappa / (2.0 * S_PI);
        T[0][0] = 0.5 + c * ti.tx * ti.tx;
        T[0][1] = c * ti.tx * ti.ty;
        T[1][0] = c * ti.ty * ti.tx;
        T[1][1] = 0.5 + c * ti.ty * ti.ty;
        rr[0][0] = ti.tx * ti.tx;
        rr[0][1] = rr[1][0] = ti.tx * ti.ty;
        rr[1][1] = ti.ty * ti.ty;
    } else {
        const double rn = rx * ti.nx + ry * ti.ny;
        const double c = -sj.w * rn / (S_PI * r2 * r2);
        T[0][0] = c * rx * rx;
        T[0][1] = c * rx * ry;
        T[1][0] = c * ry * rx;
        T[1][1] = c * ry * ry;
        rr[0][0] = rx * rx / r2;
        rr[0][1] = rr[1][0] = rx * ry / r2;
        rr[1][1] = ry * ry / r2;
    }
    // weight of log|x_i - y_j|: product integration on panels P(i) - 1, P(i), P(i) + 1
    const int Pi = i / ngl, Pj = j / ngl, ai = i % ngl, aj = j % ngl;
    int o = -1;
    if (Pj == Pi) o = 0;
    else if (Pj == (Pi + npan - 1) % npan) o = 1;
    else if (Pj == (Pi + 1) % npan) o = 2;
    double logw;
    if (o < 0) {
        logw = sj.w * 0.5 * log(r2);
    } else {
        const double mom = half * sj.spd * M[((int64_t)o * ngl + ai) * ngl + aj];
        if (i == j) {
            logw = sj.w * log(half * ti.spd) + mom;
        } else {
            const double xi0 = glx[ai] + (o == 0 ? 0.0 : (o == 1 ? 2.0 : -2.0));
            logw = sj.w * log(sqrt(r2) / fabs(xi0 - glx[aj])) + mom;
        }
    }
    const double gs = 1.0 / (4.0 * S_PI * visc);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) G[a][b] = gs * ((a == b ? -logw : 0.0) + sj.w * rr[a][b]);
    // W: w_j (I / L + e3_i e3_j^T / J), e3 = (-y, x)
    const double e3i[2] = {-ti.y, ti.x}, e3j[2] = {-sj.y, sj.x};
    const int64_t ld = 2 * (int64_t)npp;
    const int64_t base = (int64_t)s * ld * ld;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int64_t idx = base + (2 * (int64_t)j + b) * ld + 2 * i + a;
            const double wv = sj.w * ((a == b ? 1.0 / L : 0.0) + e3i[a] * e3j[b] / J);
            B0[idx] = T[a][b];
            Bw[idx] = T[a][b] + wv;
            S[idx] = G[a][b];
        }
}

__global__ void k_to_f32_stokes(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// y_P (+)= R_P B[shape(P)] R_P^T x_P for every particle P (x, y node-major, 2
// npp values per particle). CTA = 32 rows of one particle's block, as in
// block_apply.cuh, with the density turned into the body frame on load and
// the result turned back on store.
template <typename T>
__global__ void __launch_bounds__(256)
k_stokes_self(int npp, const int* __restrict__ shape_of, const T* __restrict__ B,
              const yk_particle* __restrict__ parts, const double* __restrict__ x,
              double* __restrict__ y, int acc) {
    extern __shared__ unsigned char ss_smem[];
    const int n2 = 2 * npp;
    T* xs = reinterpret_cast<T*>(ss_smem);          // n2
    T* part = xs + n2;                              // [8][32]
    const int P = blockIdx.x, r0 = blockIdx.y * 32;
    const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
    double sp, cp;
    sincos(parts[P].phi, &sp, &cp);
    const int64_t base = (int64_t)P * n2;
    for (int k = threadIdx.x; k < npp; k += blockDim.x) {
        const double sx = x[base + 2 * k], sy = x[base + 2 * k + 1];
        xs[2 * k] = (T)(cp * sx + sp * sy);
        xs[2 * k + 1] = (T)(-sp * sx + cp * sy);
    }
    __syncthreads();
    const int r = r0 + lane;
    T a = 0;
    if (r < n2) {
        const T* Mb = B + (int64_t)shape_of[P] * n2 * n2;
        for (int j = slice; j < n2; j += 8) a += Mb[(int64_t)j * n2 + r] * xs[j];
    }
    part[slice * 32 + lane] = a;
    __syncthreads();
    if (slice == 0) {
        T t = part[lane];
#pragma unroll
        for (int k = 1; k < 8; ++k) t += part[k * 32 + lane];
        part[lane] = t;
    }
    __syncthreads();
    if (slice == 0 && (lane & 1) == 0 && r < n2) {
        const double ox = (double)part[lane], oy = (double)part[lane + 1];
        const double ux = cp * ox - sp * oy, uy = sp * ox + cp * oy;
        if (acc) {
            y[base + r] += ux;
            y[base + r + 1] += uy;
        } else {
            y[base + r] = ux;
            y[base + r + 1] = uy;
        }
    }
}

// Source records: FP64 (x, y, w sigma_x, w sigma_y), FP32 (offset from the
// particle centre, w sigma).
__global__ void k_stokes_sources(int64_t n, const double* __restrict__ X,
                                 const double* __restrict__ Y, const double* __restrict__ W,
                                 const float2* __restrict__ XI, const double* __restrict__ sig,
                                 double4* __restrict__ s64, float4* __restrict__ s32) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double qx = W[i] * sig[2 * i], qy = W[i] * sig[2 * i + 1];
    if (s64) s64[i] = make_double4(X[i], Y[i], qx, qy);
    if (s32) s32[i] = make_float4(XI[i].x, XI[i].y, (float)qx, (float)qy);
}

// Pair sums over the nodes of other particles, FP64. KIND 0: traction
// -(1/pi) sum r (r . n_t)(r . q) / r^4; KIND 1: single layer
// (1/(4 pi mu)) sum (-log r q + r (r . q) / r^2). Block (target particle,
// source chunk); source particles c, c + nchunk, ...; out += (atomics).
template <int KIND>
__global__ void __launch_bounds__(FAR_TPB)
k_stokes_far64(int np, int npp, int nchunk, const double4* __restrict__ src,
               const double* __restrict__ X, const double* __restrict__ Y,
               const double* __restrict__ NX, const double* __restrict__ NY, double scale,
               double* __restrict__ out) {
    extern __shared__ double4 sf_src[];
    const int P = blockIdx.x;
    double tx[FAR_TMAX], ty[FAR_TMAX], nx[FAR_TMAX], ny[FAR_TMAX], ax[FAR_TMAX], ay[FAR_TMAX];
#pragma unroll
    for (int k = 0; k < FAR_TMAX; ++k) {
        const int t = threadIdx.x + k * FAR_TPB;
        const int64_t gi = (int64_t)P * npp + (t < npp ? t : 0);
        tx[k] = X[gi];
        ty[k] = Y[gi];
        nx[k] = KIND == 0 ? NX[gi] : 0.0;
        ny[k] = KIND == 0 ? NY[gi] : 0.0;
        ax[k] = ay[k] = 0.0;
    }
    for (int Q = blockIdx.y; Q < np; Q += nchunk) {
        if (Q == P) continue;
        __syncthreads();
        for (int s = threadIdx.x; s < npp; s += FAR_TPB) sf_src[s] = src[(int64_t)Q * npp + s];
        __syncthreads();
        for (int s = 0; s < npp; ++s) {
            const double4 q = sf_src[s];
#pragma unroll
            for (int k = 0; k < FAR_TMAX; ++k) {
                if (k * FAR_TPB >= npp) break;
                const double rx = tx[k] - q.x, ry = ty[k] - q.y;
                const double r2 = rx * rx + ry * ry;
                const double inv = 1.0 / r2;
                const double rq = rx * q.z + ry * q.w;
                if (KIND == 0) {
                    const double c = (rx * nx[k] + ry * ny[k]) * rq * inv * inv;
                    ax[k] = fma(c, rx, ax[k]);
                    ay[k] = fma(c, ry, ay[k]);
                } else {
                    const double hl = -0.5 * log(r2);
                    const double c = rq * inv;
                    ax[k] = fma(hl, q.z, fma(c, rx, ax[k]));
                    ay[k] = fma(hl, q.w, fma(c, ry, ay[k]));
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < FAR_TMAX; ++k) {
        const int t = threadIdx.x + k * FAR_TPB;
        if (t < npp) {
            const int64_t gi = (int64_t)P * npp + t;
            atomicAdd(out + 2 * gi, scale * ax[k]);
            atomicAdd(out + 2 * gi + 1, scale * ay[k]);
        }
    }
}

// The traction pair sums in FP32 (inner operator): offsets from the particle
// centres, the centre difference formed in FP64 once per particle pair, each
// source particle's sum added to FP64 accumulators.
__global__ void __launch_bounds__(FAR_TPB)
k_stokes_far32(int np, int npp, int nchunk, const float4* __restrict__ src,
               const float2* __restrict__ XI, const double* __restrict__ NX,
               const double* __restrict__ NY, const yk_particle* __restrict__ parts,
               double scale, double* __restrict__ out) {
    extern __shared__ float4 sf_src32[];
    const int P = blockIdx.x;
    float tx[FAR_TMAX], ty[FAR_TMAX], nx[FAR_TMAX], ny[FAR_TMAX];
    double ax[FAR_TMAX], ay[FAR_TMAX];
#pragma unroll
    for (int k = 0; k < FAR_TMAX; ++k) {
        const int t = threadIdx.x + k * FAR_TPB;
        const int64_t gi = (int64_t)P * npp + (t < npp ? t : 0);
        tx[k] = XI[gi].x;
        ty[k] = XI[gi].y;
        nx[k] = (float)NX[gi];
        ny[k] = (float)NY[gi];
        ax[k] = ay[k] = 0.0;
    }
    const double pcx = parts[P].cx, pcy = parts[P].cy;
    for (int Q = blockIdx.y; Q < np; Q += nchunk) {
        if (Q == P) continue;
        __syncthreads();
        for (int s = threadIdx.x; s < npp; s += FAR_TPB) sf_src32[s] = src[(int64_t)Q * npp + s];
        __syncthreads();
        const float dx = (float)(pcx - parts[Q].cx), dy = (float)(pcy - parts[Q].cy);
        float ux[FAR_TMAX], uy[FAR_TMAX], bx[FAR_TMAX], by[FAR_TMAX];
#pragma unroll
        for (int k = 0; k < FAR_TMAX; ++k) {
            ux[k] = tx[k] + dx;
            uy[k] = ty[k] + dy;
            bx[k] = by[k] = 0.0f;
        }
        for (int s = 0; s < npp; ++s) {
            const float4 q = sf_src32[s];
#pragma unroll
            for (int k = 0; k < FAR_TMAX; ++k) {
                if (k * FAR_TPB >= npp) break;
                const float rx = ux[k] - q.x, ry = uy[k] - q.y;
                const float r2 = fmaf(rx, rx, ry * ry);
                const float inv = __frcp_rn(r2);
                const float c = fmaf(rx, nx[k], ry * ny[k]) * fmaf(rx, q.z, ry * q.w) * (inv * inv);
                bx[k] = fmaf(c, rx, bx[k]);
                by[k] = fmaf(c, ry, by[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < FAR_TMAX; ++k) {
            ax[k] += bx[k];
            ay[k] += by[k];
        }
    }
#pragma unroll
    for (int k = 0; k < FAR_TMAX; ++k) {
        const int t = threadIdx.x + k * FAR_TPB;
        if (t < npp) {
            const int64_t gi = (int64_t)P * npp + t;
            atomicAdd(out + 2 * gi, scale * ax[k]);
            atomicAdd(out + 2 * gi + 1, scale * ay[k]);
        }
    }
}

// Per particle: L = sum w, J = sum w |x - a|^2 (world frame).
__global__ void k_particle_LJ(int npp, const double* __restrict__ X, const double* __restrict__ Y,
                              const double* __restrict__ W, const yk_particle* __restrict__ parts,
                              double* __restrict__ LJ) {
    const int P = blockIdx.x;
    const double cx = parts[P].cx, cy = parts[P].cy;
    double l = 0.0, j = 0.0;
    for (int k = threadIdx.x; k < npp; k += blockDim.x) {
        const int64_t i = (int64_t)P * npp + k;
        const double dx = X[i] - cx, dy = Y[i] - cy;
        l += W[i];
        j += W[i] * (dx * dx + dy * dy);
    }
    __shared__ double rl[256], rj[256];
    rl[threadIdx.x] = l;
    rj[threadIdx.x] = j;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            rl[threadIdx.x] += rl[threadIdx.x + o];
            rj[threadIdx.x] += rj[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        LJ[2 * P] = rl[0];
        LJ[2 * P + 1] = rj[0];
    }
}

// sigma_inc = F_P / L_P + tau_P (x - a_P)^perp / J_P
__global__ void k_incident(int64_t n, int npp, const double* __restrict__ F,
                           const double* __restrict__ tau, const double* __restrict__ LJ,
                           const double* __restrict__ X, const double* __restrict__ Y,
                           const yk_particle* __restrict__ parts, double* __restrict__ s) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int P = (int)(i / npp);
    const double dx = X[i] - parts[P].cx, dy = Y[i] - parts[P].cy;
    const double t = tau[P] / LJ[2 * P + 1], il = 1.0 / LJ[2 * P];
    s[2 * i] = F[2 * P] * il - t * dy;
    s[2 * i + 1] = F[2 * P + 1] * il + t * dx;
}

// out = a - b (2n values)
__global__ void k_stokes_sub(int64_t n2, const double* __restrict__ a, const double* __restrict__ b,
                             double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n2) out[i] = a[i] - b[i];
}

__global__ void k_stokes_add(int64_t n2, const double* __restrict__ a,
                             const double* __restrict__ b, double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n2) out[i] = a[i] + b[i];
}

// Eq. mobilityu's averages: v_P = sum w u / L_P, omega_P = sum w (x - a) x u / J_P.
__global__ void k_rigid_average(int npp, const double* __restrict__ u, const double* __restrict__ X,
                                const double* __restrict__ Y, const double* __restrict__ W,
                                const yk_particle* __restrict__ parts,
                                const double* __restrict__ LJ, double* __restrict__ v,
                                double* __restrict__ om) {
    const int P = blockIdx.x;
    const double cx = parts[P].cx, cy = parts[P].cy;
    double sx = 0.0, sy = 0.0, so = 0.0;
    for (int k = threadIdx.x; k < npp; k += blockDim.x) {
        const int64_t i = (int64_t)P * npp + k;
        const double ux = u[2 * i], uy = u[2 * i + 1];
        sx += W[i] * ux;
        sy += W[i] * uy;
        so += W[i] * ((X[i] - cx) * uy - (Y[i] - cy) * ux);
    }
    __shared__ double r[3][256];
    r[0][threadIdx.x] = sx;
    r[1][threadIdx.x] = sy;
    r[2][threadIdx.x] = so;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int c = 0; c < 3; ++c) r[c][threadIdx.x] += r[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        v[2 * P] = r[0][0] / LJ[2 * P];
        v[2 * P + 1] = r[1][0] / LJ[2 * P];
        om[P] = r[2][0] / LJ[2 * P + 1];
    }
}

// ---------------------------------------------------------------------------

void stokes_free(yk_geom* g) {
    Stokes& S = g->stokes;
    cudaStream_t st = g->ctx->stream;
    void* bufs[] = {S.B0, S.Bw, S.Bw32, S.S, S.moments, S.shapeLJ, S.LJ, S.s64, S.s32,
                    S.sinc, S.mu, S.rhs, S.tmp, S.u, S.vo};
    for (void* b : bufs) dev_free(b, st);
    free_workspace(S.ws, st);
    S = Stokes{};
}

// Blocks, moments and buffers, on the first Stokes call of a geometry (the
// shapes of a geometry never change).
static int stokes_ready(yk_geom* g) {
    Stokes& S = g->stokes;
    if (S.ready) return YK_OK;
    if (g->npan < 3 || g->ngl > 64 || g->npp > FAR_TPB * FAR_TMAX) return YK_ERR_ARG;
    cudaStream_t st = g->ctx->stream;
    const int npp = g->npp, ns = g->nshape;
    const int64_t ld = 2 * (int64_t)npp, blk = ld * ld;
    const int64_t n2 = 2 * g->n;
    YK_TRY(dev_alloc((void**)&S.B0, sizeof(double) * blk * ns, st));
    YK_TRY(dev_alloc((void**)&S.Bw, sizeof(double) * blk * ns, st));
    YK_TRY(dev_alloc((void**)&S.Bw32, sizeof(float) * blk * ns, st));
    YK_TRY(dev_alloc((void**)&S.S, sizeof(double) * blk * ns, st));
    YK_TRY(dev_alloc((void**)&S.moments, sizeof(double) * 3 * g->ngl * g->ngl, st));
    YK_TRY(dev_alloc((void**)&S.shapeLJ, sizeof(double) * 2 * ns, st));
    YK_TRY(dev_alloc((void**)&S.LJ, sizeof(double) * 2 * g->np, st));
    YK_TRY(dev_alloc((void**)&S.s64, sizeof(double4) * g->n, st));
    YK_TRY(dev_alloc((void**)&S.s32, sizeof(float4) * g->n, st));
    for (double** v : {&S.sinc, &S.mu, &S.rhs, &S.tmp, &S.u})
        YK_TRY(dev_alloc((void**)v, sizeof(double) * n2, st));
    YK_TRY(dev_alloc((void**)&S.vo, sizeof(double) * 3 * g->np, st));
    YK_TRY(alloc_krylov(S.ws, n2, g->prm.gmres_restart, st));
    YK_LAUNCH(k_log_moments, 3 * g->ngl, 64, 0, st, g->ngl, g->d_glx, S.moments);
    YK_LAUNCH(k_shape_LJ, ns, 256, 0, st, g->npan, g->ngl, g->d_shape_ab, g->d_glx, g->d_glw,
              S.shapeLJ);
    YK_LAUNCH(k_stokes_blocks, dim3(ceil_div((int64_t)npp * npp, 256), ns), 256, 0, st, g->npan,
              g->ngl, g->prm.viscosity, g->d_shape_ab, g->d_glx, g->d_glw, S.moments, S.shapeLJ,
              S.B0, S.Bw, S.S);
    YK_LAUNCH(k_to_f32_stokes, ceil_div(blk * ns, 256), 256, 0, st, blk * ns, S.Bw, S.Bw32);
    YK_TRY_CUDA(cudaGetLastError());
    S.ready = true;
    return YK_OK;
}

static int far_chunks(const yk_geom* g) {
    return std::max(1, std::min(g->np - 1, ceil_div(4 * 152, g->np)));
}

int stokes_apply(yk_geom* g, const double* sig, double* out, Prec prec, int which) {
    YK_TRY(stokes_ready(g));
    Stokes& S = g->stokes;
    cudaStream_t st = g->ctx->stream;
    const int npp = g->npp, np = g->np;
    const bool f32 = prec == Prec::F32 && which == STOKES_COMPLETED;
    const dim3 sgrid(np, ceil_div(2 * npp, 32));
    if (which == STOKES_VELOCITY) {
        YK_LAUNCH(k_stokes_self<double>, sgrid, 256, sizeof(double) * (2 * npp + 256), st, npp,
                  g->d_shape_of, S.S, g->d_particles, sig, out, 0);
    } else if (f32) {
        YK_LAUNCH(k_stokes_self<float>, sgrid, 256, sizeof(float) * (2 * npp + 256), st, npp,
                  g->d_shape_of, S.Bw32, g->d_particles, sig, out, 0);
    } else {
        YK_LAUNCH(k_stokes_self<double>, sgrid, 256, sizeof(double) * (2 * npp + 256), st, npp,
                  g->d_shape_of, which == STOKES_COMPLETED ? S.Bw : S.B0, g->d_particles, sig,
                  out, 0);
    }
    if (np < 2) return YK_OK;
    YK_LAUNCH(k_stokes_sources, ceil_div(g->n, 256), 256, 0, st, g->n, g->d_x, g->d_y, g->d_w,
              g->d_xi, sig, f32 ? nullptr : S.s64, f32 ? S.s32 : nullptr);
    const dim3 fgrid(np, far_chunks(g));
    if (f32) {
        YK_LAUNCH(k_stokes_far32, fgrid, FAR_TPB, sizeof(float4) * npp, st, np, npp, (int)fgrid.y,
                  S.s32, g->d_xi, g->d_nx, g->d_ny, g->d_particles, -1.0 / S_PI, out);
    } else if (which == STOKES_VELOCITY) {
        YK_LAUNCH(k_stokes_far64<1>, fgrid, FAR_TPB, sizeof(double4) * npp, st, np, npp,
                  (int)fgrid.y, S.s64, g->d_x, g->d_y, g->d_nx, g->d_ny,
                  1.0 / (4.0 * S_PI * g->prm.viscosity), out);
    } else {
        YK_LAUNCH(k_stokes_far64<0>, fgrid, FAR_TPB, sizeof(double4) * npp, st, np, npp,
                  (int)fgrid.y, S.s64, g->d_x, g->d_y, g->d_nx, g->d_ny, -1.0 / S_PI, out);
    }
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

int mobility(yk_geom* g, const double* F, const double* tau, double* v, double* omega,
             double* sigma_out, yk_solve_info* info) {
    YK_TRY(stokes_ready(g));
    Stokes& S = g->stokes;
    cudaStream_t st = g->ctx->stream;
    const int64_t n2 = 2 * g->n;
    const int nb = ceil_div(n2, 256);
    YK_LAUNCH(k_particle_LJ, g->np, 256, 0, st, g->npp, g->d_x, g->d_y, g->d_w, g->d_particles,
              S.LJ);
    YK_LAUNCH(k_incident, ceil_div(g->n, 256), 256, 0, st, g->n, g->npp, F, tau, S.LJ, g->d_x,
              g->d_y, g->d_particles, S.sinc);
    // rhs = -(1/2 I + K*) sigma_inc = sigma_inc - (1/2 I + K* + W) sigma_inc, since
    // sigma_inc lies in the span of the rigid motions (W sigma_inc = sigma_inc)
    YK_TRY(stokes_apply(g, S.sinc, S.tmp, Prec::F64, STOKES_COMPLETED));
    YK_LAUNCH(k_stokes_sub, nb, 256, 0, st, n2, S.sinc, S.tmp, S.rhs);
    KrylovOp op;
    op.ctx = g->ctx;
    op.ws = &S.ws;
    op.n = n2;
    op.apply = [g](const double* x, double* y, Prec p) {
        return stokes_apply(g, x, y, p == Prec::F32 ? Prec::F32 : Prec::F64, STOKES_COMPLETED);
    };
    const int rc = solve_op(op, g->prm, Prec::F64, S.rhs, S.mu, nullptr, info);
    if (rc != YK_OK && rc != YK_ERR_NOT_CONVERGED) return rc;
    double* sig = sigma_out ? sigma_out : S.tmp;
    YK_LAUNCH(k_stokes_add, nb, 256, 0, st, n2, S.sinc, S.mu, sig);
    YK_TRY(stokes_apply(g, sig, S.u, Prec::F64, STOKES_VELOCITY));
    YK_LAUNCH(k_rigid_average, g->np, 256, 0, st, g->npp, S.u, g->d_x, g->d_y, g->d_w,
              g->d_particles, S.LJ, v, omega);
    YK_TRY_CUDA(cudaGetLastError());
    return rc;
}

}  // namespace yk
