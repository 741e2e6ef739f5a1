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
//   * other particles: node-by-node sums for near particle pairs (FP64
//     (x, y, w sigma) records, or FP32 offsets from each particle's centre with
//     the centre difference formed in FP64 for the inner operator; one block
//     per target particle), complex-variable particle expansions for far pairs
//     (multipoles, translation to local expansions, evaluation; FP64, or FP32
//     for the inner operator), over pair lists built once per configuration;
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
constexpr double FAR_FACTOR = 2.0; // particle expansions beyond 2 (r_P + r_Q) between centres
constexpr int STOKES_MAX_PARTICLES = 16384;   // the pair lists hold every particle pair
constexpr int SP = 40;            // largest order of the particle expansions
constexpr int SP1 = SP + 1;

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

// ---------------------------------------------------------------------------
// Particle pairs. A pair whose centres are at least 2 (r_P + r_Q) apart (r
// the bounding radius) is far: its interaction goes through the particle
// expansions below; the others are summed node by node. The lists (near
// partners and far pairs per target particle, CSR) are built once per
// configuration, in FP64, so that both sides take the same decision.
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool stokes_far_pair(const yk_particle& P, const yk_particle& Q,
                                                double* dist) {
    const double dx = P.cx - Q.cx, dy = P.cy - Q.cy;
    *dist = sqrt(dx * dx + dy * dy);
    return *dist >= FAR_FACTOR * (fmax(P.A, P.B) + fmax(Q.A, Q.B));
}

// smallest order with (max r / (|z0| - max r))^(p - 1) below eps = e^le
__device__ __forceinline__ int stokes_order(double dist, double rm, double le) {
    const double q = rm / (dist - rm);
    return min(max((int)ceil(le / log(q)) + 1, 2), SP);
}

// One warp per particle P, lanes over Q; entries in order of Q.
__global__ void k_stokes_count(int np, const yk_particle* __restrict__ parts,
                               int* __restrict__ nnear, int* __restrict__ nfar) {
    const int P = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (P >= np) return;   // warp-uniform
    const yk_particle pp = parts[P];
    int cn = 0, cf = 0;
    for (int Q0 = 0; Q0 < np; Q0 += 32) {
        const int Q = Q0 + lane;
        bool isn = false, isf = false;
        if (Q < np && Q != P) {
            double d;
            isf = stokes_far_pair(pp, parts[Q], &d);
            isn = !isf;
        }
        cn += __popc(__ballot_sync(0xffffffffu, isn));
        cf += __popc(__ballot_sync(0xffffffffu, isf));
    }
    if (lane == 0) {
        nnear[P] = cn;
        nfar[P] = cf;
    }
}

__global__ void k_stokes_fill(int np, const yk_particle* __restrict__ parts,
                              const int* __restrict__ near_off, int* __restrict__ near_idx,
                              const int* __restrict__ far_off, StokesFar* __restrict__ far) {
    const int P = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (P >= np) return;   // warp-uniform
    const yk_particle pp = parts[P];
    int in = near_off[P], jf = far_off[P];
    for (int Q0 = 0; Q0 < np; Q0 += 32) {
        const int Q = Q0 + lane;
        bool isn = false, isf = false;
        double d = 0.0;
        yk_particle qq;
        if (Q < np && Q != P) {
            qq = parts[Q];
            isf = stokes_far_pair(pp, qq, &d);
            isn = !isf;
        }
        const unsigned lt = (1u << lane) - 1u;
        const unsigned mn = __ballot_sync(0xffffffffu, isn);
        const unsigned mf = __ballot_sync(0xffffffffu, isf);
        if (isn) near_idx[in + __popc(mn & lt)] = Q;
        if (isf) {
            StokesFar e;
            e.z0 = make_double2(pp.cx - qq.cx, pp.cy - qq.cy);
            const double id = 1.0 / (d * d);
            e.zi = make_double2(e.z0.x * id, -e.z0.y * id);
            e.logd = log(d);
            e.q = Q;
            const double rm = fmax(fmax(pp.A, pp.B), fmax(qq.A, qq.B));
            e.p64 = (short)stokes_order(d, rm, -39.14);    // 1e-17
            e.p32 = (short)stokes_order(d, rm, -18.42);    // 1e-8
            far[jf + __popc(mf & lt)] = e;
        }
        in += __popc(mn);
        jf += __popc(mf);
    }
}

// 1 / x for x > 0 in the float range: FP32 estimate and two Newton steps
__device__ __forceinline__ double recip(double x) {
    double r = (double)__frcp_rn((float)x);
    r = fma(r, fma(-x, r, 1.0), r);
    return fma(r, fma(-x, r, 1.0), r);
}

// Node-by-node sums over the near particles, FP64. KIND 0: traction
// -(1/pi) sum r (r . n_t)(r . q) / r^4; KIND 1: single layer
// (1/(4 pi mu)) sum (-log r q + r (r . q) / r^2). Block = target particle,
// blockDim a multiple of 32 covering npp (up to FAR_TMAX targets a thread).
template <int KIND>
__global__ void __launch_bounds__(FAR_TPB)
k_stokes_near64(int npp, const int* __restrict__ near_off, const int* __restrict__ near_idx,
                const double4* __restrict__ src, const double* __restrict__ X,
                const double* __restrict__ Y, const double* __restrict__ NX,
                const double* __restrict__ NY, double scale, double* __restrict__ out) {
    extern __shared__ double4 sf_src[];
    const int P = blockIdx.x;
    const int e0 = near_off[P], e1 = near_off[P + 1];
    if (e0 == e1) return;
    const int tpb = blockDim.x;
    double tx[FAR_TMAX], ty[FAR_TMAX], nx[FAR_TMAX], ny[FAR_TMAX], ax[FAR_TMAX], ay[FAR_TMAX];
#pragma unroll
    for (int k = 0; k < FAR_TMAX; ++k) {
        const int t = threadIdx.x + k * tpb;
        const int64_t gi = (int64_t)P * npp + (t < npp ? t : 0);
        tx[k] = X[gi];
        ty[k] = Y[gi];
        nx[k] = KIND == 0 ? NX[gi] : 0.0;
        ny[k] = KIND == 0 ? NY[gi] : 0.0;
        ax[k] = ay[k] = 0.0;
    }
    for (int e = e0; e < e1; ++e) {
        const int Q = near_idx[e];
        __syncthreads();
        for (int s = threadIdx.x; s < npp; s += tpb) sf_src[s] = src[(int64_t)Q * npp + s];
        __syncthreads();
        for (int s = 0; s < npp; ++s) {
            const double4 q = sf_src[s];
#pragma unroll
            for (int k = 0; k < FAR_TMAX; ++k) {
                if (k * tpb >= npp) break;
                const double rx = tx[k] - q.x, ry = ty[k] - q.y;
                const double r2 = rx * rx + ry * ry;
                const double inv = recip(r2);
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
        const int t = threadIdx.x + k * tpb;
        if (t < npp) {
            const int64_t gi = (int64_t)P * npp + t;
            out[2 * gi] += scale * ax[k];
            out[2 * gi + 1] += scale * ay[k];
        }
    }
}

// The traction node-by-node sums over the near particles in FP32 (inner
// operator): offsets from the particle centres, the centre difference formed
// in FP64 once per particle pair, each source particle's sum added to FP64
// accumulators.
__global__ void __launch_bounds__(FAR_TPB)
k_stokes_near32(int npp, const int* __restrict__ near_off, const int* __restrict__ near_idx,
                const float4* __restrict__ src, const float2* __restrict__ XI,
                const double* __restrict__ NX, const double* __restrict__ NY,
                const yk_particle* __restrict__ parts, double scale, double* __restrict__ out) {
    extern __shared__ float4 sf_src32[];
    __shared__ float2 dq;
    const int P = blockIdx.x;
    const int e0 = near_off[P], e1 = near_off[P + 1];
    if (e0 == e1) return;
    const int tpb = blockDim.x;
    float tx[FAR_TMAX], ty[FAR_TMAX], nx[FAR_TMAX], ny[FAR_TMAX];
    double ax[FAR_TMAX], ay[FAR_TMAX];
#pragma unroll
    for (int k = 0; k < FAR_TMAX; ++k) {
        const int t = threadIdx.x + k * tpb;
        const int64_t gi = (int64_t)P * npp + (t < npp ? t : 0);
        tx[k] = XI[gi].x;
        ty[k] = XI[gi].y;
        nx[k] = (float)NX[gi];
        ny[k] = (float)NY[gi];
        ax[k] = ay[k] = 0.0;
    }
    for (int e = e0; e < e1; ++e) {
        const int Q = near_idx[e];
        __syncthreads();
        for (int s = threadIdx.x; s < npp; s += tpb) sf_src32[s] = src[(int64_t)Q * npp + s];
        if (threadIdx.x == 0)
            dq = make_float2((float)(parts[P].cx - parts[Q].cx), (float)(parts[P].cy - parts[Q].cy));
        __syncthreads();
        float ux[FAR_TMAX], uy[FAR_TMAX], bx[FAR_TMAX], by[FAR_TMAX];
#pragma unroll
        for (int k = 0; k < FAR_TMAX; ++k) {
            ux[k] = tx[k] + dq.x;
            uy[k] = ty[k] + dq.y;
            bx[k] = by[k] = 0.0f;
        }
        for (int s = 0; s < npp; ++s) {
            const float4 q = sf_src32[s];
#pragma unroll
            for (int k = 0; k < FAR_TMAX; ++k) {
                if (k * tpb >= npp) break;
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
        const int t = threadIdx.x + k * tpb;
        if (t < npp) {
            const int64_t gi = (int64_t)P * npp + t;
            out[2 * gi] += scale * ax[k];
            out[2 * gi + 1] += scale * ay[k];
        }
    }
}

// ---------------------------------------------------------------------------
// Particle expansions of the far pairs (FP64 for the accurate operator, FP32
// for the inner one). With z = x + i y, f = w (sigma_x + i sigma_y) at
// s = y - c_Q and w = z - c_Q, the single layer and its traction summed over
// the sources of Q are (complex forms of the stokeslet and of its stress)
//   4 pi mu u = -(1/2) Phi_A(w) - (1/2) conj(Phi_Bc(w)) + (1/2) A_0
//               + (1/2) w conj(Phi_A'(w)) - (1/2) conj(Psi_D'(w)),
//   -4 pi t   = conj(nu) [conj(Phi_Bc'(w)) + conj(Psi_D''(w)) - w conj(Phi_A''(w))]
//               + nu [conj(Phi_A'(w)) + Phi_A'(w)],
// with the 2-D Laplace log-multipoles
//   Phi_A  = A_0 log w - sum_k A_k w^-k / k,              A_k = sum f s^k,
//   Phi_Bc = conj(A_0) log w - sum_k conj(B_k) w^-k / k,  B_k = sum f conj(s)^k,
//   Psi_D  = conj(D_0) log w - sum_k conj(D_k) w^-k / k,  D_k = sum conj(f) s conj(s)^k.
// Each is shifted to a local expansion about the target particle's centre
// (the Laplace multipole-to-local translation). The factor w = omega + z0
// (z0 = c_P - c_Q) is carried by a fourth local series conj(z0) Phi_A, so no
// large absolute coordinate enters, and the constant (1/2) A_0 is folded into
// the first. Only log|z0| enters the constant terms (their imaginary parts
// cancel in u). The order per pair is the smallest that brings
// (max r / (|z0| - max r))^p to 1e-17 (FP64) or 1e-8 (FP32).
// ---------------------------------------------------------------------------

template <typename T>
struct cx {
    T x, y;
};
template <typename T>
__device__ __forceinline__ cx<T> mk(T a, T b) {
    cx<T> r;
    r.x = a;
    r.y = b;
    return r;
}
template <typename T>
__device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) {
    return mk<T>(a.x + b.x, a.y + b.y);
}
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) {
    return mk<T>(a.x - b.x, a.y - b.y);
}
template <typename T>
__device__ __forceinline__ cx<T> operator*(cx<T> a, T s) {
    return mk<T>(a.x * s, a.y * s);
}
template <typename T>
__device__ __forceinline__ cx<T> cj(cx<T> a) {
    return mk<T>(a.x, -a.y);
}
template <typename T>
__device__ cx<T> cpow(cx<T> a, int k) {
    cx<T> r = mk<T>(1, 0);
    while (k) {
        if (k & 1) r = r * a;
        a = a * a;
        k >>= 1;
    }
    return r;
}

// Multipole coefficients coef[Q][set][k] (sets Phi_A, Phi_Bc, Psi_D) of every
// particle, up to order kmax. Block Q, thread (set, k).
template <typename T>
__global__ void k_stokes_p2m(int npp, int kmax, const double4* __restrict__ s64,
                             const float4* __restrict__ s32, const yk_particle* __restrict__ parts,
                             cx<T>* __restrict__ coef) {
    const int Q = blockIdx.x, t = threadIdx.x;
    if (t >= 3 * SP1) return;
    const int set = t / SP1, k = t % SP1;
    cx<T> acc = mk<T>(0, 0);
    if (k <= kmax) {
        const double cxq = parts[Q].cx, cyq = parts[Q].cy;
        for (int j = 0; j < npp; ++j) {
            cx<T> sv, f;
            if (sizeof(T) == 8) {
                const double4 r = s64[(int64_t)Q * npp + j];
                sv = mk<T>((T)(r.x - cxq), (T)(r.y - cyq));
                f = mk<T>((T)r.z, (T)r.w);
            } else {
                const float4 r = s32[(int64_t)Q * npp + j];
                sv = mk<T>((T)r.x, (T)r.y);
                f = mk<T>((T)r.z, (T)r.w);
            }
            if (set == 0) acc = acc + f * cpow(sv, k);
            else if (set == 1) acc = acc + f * cpow(cj(sv), k);
            else acc = acc + cj(f) * sv * cpow(cj(sv), k);
        }
    }
    cx<T> a = set == 0 ? acc : cj(acc);
    if (k > 0) a = a * (T)(-1.0 / k);
    coef[((int64_t)Q * 3 + set) * SP1 + k] = a;
}

// Local coefficients loc[P][set][l] (sets Phi_A, Phi_Bc, Psi_D, conj(z0)
// Phi_A) of every particle from its far pairs; lmax[P] = the largest order
// used (0: no far pair). Block P; each half-warp takes a far pair (the 16
// half-warps of the block take pairs h, h + 16, ...), lane l of the half
// the orders l, l + 16, l + 32 up to the pair's order, so that two pairs of
// order below 16 share a warp instruction on the FP64 pipe.
template <typename T>
__global__ void __launch_bounds__(256)
k_stokes_m2l(const int* __restrict__ far_off, const StokesFar* __restrict__ far,
             const cx<T>* __restrict__ coef, cx<T>* __restrict__ loc, int* __restrict__ lmax) {
    __shared__ cx<T> red[8][4 * SP1];
    __shared__ T invk[SP1 + 1];
    __shared__ int wmax[8];
    const int P = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int hl = lane & 15, half = lane >> 4;
    for (int k = threadIdx.x; k <= SP1; k += blockDim.x) invk[k] = k ? (T)(1.0 / k) : (T)0;
    __syncthreads();
    constexpr int R = (SP + 16) / 16;                // rounds of 16 orders
    cx<T> acc[R][4];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[r][s] = mk<T>(0, 0);
    int pm = 0;
    for (int e = far_off[P] + 2 * warp + half; e < far_off[P + 1]; e += 16) {
        const StokesFar E = far[e];
        const int p = sizeof(T) == 8 ? E.p64 : E.p32;
        pm = max(pm, p);
        const cx<T>* a = coef + (int64_t)E.q * 3 * SP1;
        const cx<T> zi = mk<T>((T)E.zi.x, (T)E.zi.y);
        const cx<T> z0c = mk<T>((T)E.z0.x, (T)(-E.z0.y));
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int l = hl + 16 * r;
            if (l > p) break;
            cx<T> v[3];
            if (l == 0) {
                const T lg = (T)E.logd;
                cx<T> zk = zi;
#pragma unroll
                for (int s = 0; s < 3; ++s) v[s] = a[s * SP1] * lg;
                for (int k = 1; k <= p; ++k) {
#pragma unroll
                    for (int s = 0; s < 3; ++s) v[s] = v[s] + a[s * SP1 + k] * zk;
                    zk = zk * zi;
                }
            } else {
                const T il = invk[l];
#pragma unroll
                for (int s = 0; s < 3; ++s) v[s] = a[s * SP1] * (-il);
                cx<T> zk = zi;
                T c = 1;                                   // C(k + l - 1, l) at k = 1
                for (int k = 1; k <= p; ++k) {
                    const cx<T> w = zk * c;
#pragma unroll
                    for (int s = 0; s < 3; ++s) v[s] = v[s] + a[s * SP1 + k] * w;
                    zk = zk * zi;
                    c = c * (T)(k + l) * invk[k];
                }
                const cx<T> zl = cpow(zi, l) * (T)((l & 1) ? -1 : 1);
#pragma unroll
                for (int s = 0; s < 3; ++s) v[s] = v[s] * zl;
            }
            acc[r][3] = acc[r][3] + z0c * v[0];
            if (l == 0) v[0] = v[0] - a[0];
#pragma unroll
            for (int s = 0; s < 3; ++s) acc[r][s] = acc[r][s] + v[s];
        }
    }
    // the two halves hold the same orders: add them, then the warps in smem
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            acc[r][s].x += __shfl_xor_sync(0xffffffffu, acc[r][s].x, 16);
            acc[r][s].y += __shfl_xor_sync(0xffffffffu, acc[r][s].y, 16);
        }
    if (half == 0)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int l = hl + 16 * r;
            if (l <= SP)
#pragma unroll
                for (int s = 0; s < 4; ++s) red[warp][s * SP1 + l] = acc[r][s];
        }
    for (int o = 16; o > 0; o >>= 1) pm = max(pm, __shfl_xor_sync(0xffffffffu, pm, o));
    if (lane == 0) wmax[warp] = pm;
    __syncthreads();
    for (int e = threadIdx.x; e < 4 * SP1; e += blockDim.x) {
        cx<T> t = red[0][e];
        for (int w = 1; w < 8; ++w) t = t + red[w][e];
        loc[(int64_t)P * 4 * SP1 + e] = t;
    }
    if (threadIdx.x == 0) {
        int m = 0;
        for (int w = 0; w < 8; ++w) m = max(m, wmax[w]);
        lmax[P] = m;
    }
}

// value, first and second derivative of sum_{l <= n} b_l w^l
template <typename T>
__device__ __forceinline__ void horner2(const cx<T>* b, int n, cx<T> w, cx<T>& f, cx<T>& f1,
                                        cx<T>& f2) {
    f = b[n];
    f1 = mk<T>(0, 0);
    f2 = mk<T>(0, 0);
    for (int l = n - 1; l >= 0; --l) {
        f2 = f2 * w + f1 * (T)2;
        f1 = f1 * w + f;
        f = f * w + b[l];
    }
}

// out += the far field of the local expansions at every node (KIND 0:
// traction with the node's normal, KIND 1: velocity). Block P.
template <typename T, int KIND>
__global__ void k_stokes_l2p(int npp, const double* __restrict__ X, const double* __restrict__ Y,
                             const float2* __restrict__ XI, const double* __restrict__ NX,
                             const double* __restrict__ NY, const yk_particle* __restrict__ parts,
                             const cx<T>* __restrict__ loc, const int* __restrict__ lmax,
                             double visc, double* __restrict__ out) {
    __shared__ cx<T> b[4 * SP1];
    const int P = blockIdx.x;
    const int n = lmax[P];
    if (n == 0) return;
    for (int e = threadIdx.x; e < 4 * SP1; e += blockDim.x) b[e] = loc[(int64_t)P * 4 * SP1 + e];
    __syncthreads();
    const double pcx = parts[P].cx, pcy = parts[P].cy;
    for (int t = threadIdx.x; t < npp; t += blockDim.x) {
        const int64_t i = (int64_t)P * npp + t;
        const cx<T> w = sizeof(T) == 8 ? mk<T>((T)(X[i] - pcx), (T)(Y[i] - pcy))
                                       : mk<T>((T)XI[i].x, (T)XI[i].y);
        cx<T> A, A1, A2, B, B1, B2, D, D1, D2, C, C1, C2;
        horner2(b, n, w, A, A1, A2);
        horner2(b + SP1, n, w, B, B1, B2);
        horner2(b + 2 * SP1, n, w, D, D1, D2);
        horner2(b + 3 * SP1, n, w, C, C1, C2);
        double rx, ry;
        if (KIND == 1) {
            // 4 pi mu u = -(A + conj B)/2 + (w conj A' + conj C')/2 - conj D'/2
            const cx<T> wa = w * cj(A1);
            rx = 0.5 * (double)(-A.x - B.x + wa.x + C1.x - D1.x);
            ry = 0.5 * (double)(-A.y + B.y + wa.y - C1.y + D1.y);
            const double sc = 1.0 / (4.0 * S_PI * visc);
            rx *= sc;
            ry *= sc;
        } else {
            // -4 pi t = conj(nu) (conj B' + conj D'' - w conj A'' - conj C'') + nu (conj A' + A')
            const cx<T> nu = mk<T>((T)NX[i], (T)NY[i]);
            const cx<T> h = cj(B1 + D2 - C2) - w * cj(A2);
            const cx<T> s1 = cj(nu) * h + nu * (A1.x * (T)2);
            rx = -(double)s1.x / (4.0 * S_PI);
            ry = -(double)s1.y / (4.0 * S_PI);
        }
        out[2 * i] += rx;
        out[2 * i + 1] += ry;
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
                    S.sinc, S.mu, S.rhs, S.tmp, S.u, S.vo, S.coef64, S.loc64, S.coef32,
                    S.loc32, S.lmax64, S.lmax32, S.near_off, S.near_idx, S.far_off, S.far};
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
    const int npp = g->npp, ns = g->nshape, np = g->np;
    const int64_t ld = 2 * (int64_t)npp, blk = ld * ld;
    const int64_t n2 = 2 * g->n;
    YK_TRY(dev_alloc((void**)&S.B0, sizeof(double) * blk * ns, st));
    YK_TRY(dev_alloc((void**)&S.Bw, sizeof(double) * blk * ns, st));
    YK_TRY(dev_alloc((void**)&S.Bw32, sizeof(float) * blk * ns, st));
    YK_TRY(dev_alloc((void**)&S.S, sizeof(double) * blk * ns, st));
    YK_TRY(dev_alloc((void**)&S.moments, sizeof(double) * 3 * g->ngl * g->ngl, st));
    YK_TRY(dev_alloc((void**)&S.shapeLJ, sizeof(double) * 2 * ns, st));
    YK_TRY(dev_alloc((void**)&S.LJ, sizeof(double) * 2 * np, st));
    YK_TRY(dev_alloc((void**)&S.s64, sizeof(double4) * g->n, st));
    YK_TRY(dev_alloc((void**)&S.s32, sizeof(float4) * g->n, st));
    for (double** v : {&S.sinc, &S.mu, &S.rhs, &S.tmp, &S.u})
        YK_TRY(dev_alloc((void**)v, sizeof(double) * n2, st));
    YK_TRY(dev_alloc((void**)&S.vo, sizeof(double) * 3 * np, st));
    YK_TRY(dev_alloc((void**)&S.coef64, sizeof(double2) * 3 * SP1 * np, st));
    YK_TRY(dev_alloc((void**)&S.loc64, sizeof(double2) * 4 * SP1 * np, st));
    YK_TRY(dev_alloc((void**)&S.coef32, sizeof(float2) * 3 * SP1 * np, st));
    YK_TRY(dev_alloc((void**)&S.loc32, sizeof(float2) * 4 * SP1 * np, st));
    YK_TRY(dev_alloc((void**)&S.lmax64, sizeof(int) * np, st));
    YK_TRY(dev_alloc((void**)&S.lmax32, sizeof(int) * np, st));
    YK_TRY(dev_alloc((void**)&S.near_off, sizeof(int) * (np + 1), st));
    YK_TRY(dev_alloc((void**)&S.far_off, sizeof(int) * (np + 1), st));
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

// Near partners and far pairs of every particle (CSR), for the current
// positions: counts, prefix sums on the host, fill.
static int stokes_lists(yk_geom* g) {
    Stokes& S = g->stokes;
    if (S.lists_valid) return YK_OK;
    if (g->np > STOKES_MAX_PARTICLES) return YK_ERR_TOO_LARGE;   // pair lists ~ 48 np^2 bytes
    cudaStream_t st = g->ctx->stream;
    const int np = g->np;
    std::vector<int> cn(np), cf(np);
    YK_LAUNCH(k_stokes_count, ceil_div(np, 4), 128, 0, st, np, g->d_particles, S.near_off,
              S.far_off);
    YK_TRY_CUDA(cudaMemcpyAsync(cn.data(), S.near_off, sizeof(int) * np, cudaMemcpyDeviceToHost, st));
    YK_TRY_CUDA(cudaMemcpyAsync(cf.data(), S.far_off, sizeof(int) * np, cudaMemcpyDeviceToHost, st));
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    std::vector<int> on(np + 1, 0), of(np + 1, 0);
    for (int i = 0; i < np; ++i) {
        on[i + 1] = on[i] + cn[i];
        of[i + 1] = of[i] + cf[i];
    }
    if (on[np] > S.near_cap) {
        dev_free(S.near_idx, st);
        S.near_idx = nullptr;
        YK_TRY(dev_alloc((void**)&S.near_idx, sizeof(int) * std::max(1, on[np]), st));
        S.near_cap = on[np];
    }
    if (of[np] > S.far_cap) {
        dev_free(S.far, st);
        S.far = nullptr;
        YK_TRY(dev_alloc((void**)&S.far, sizeof(StokesFar) * std::max(1, of[np]), st));
        S.far_cap = of[np];
    }
    YK_TRY_CUDA(cudaMemcpyAsync(S.near_off, on.data(), sizeof(int) * (np + 1),
                                cudaMemcpyHostToDevice, st));
    YK_TRY_CUDA(cudaMemcpyAsync(S.far_off, of.data(), sizeof(int) * (np + 1),
                                cudaMemcpyHostToDevice, st));
    YK_LAUNCH(k_stokes_fill, ceil_div(np, 4), 128, 0, st, np, g->d_particles, S.near_off,
              S.near_idx, S.far_off, S.far);
    YK_TRY_CUDA(cudaStreamSynchronize(st));   // the host vectors go out of scope
    S.lists_valid = true;
    return YK_OK;
}

int stokes_apply(yk_geom* g, const double* sig, double* out, Prec prec, int which) {
    YK_TRY(stokes_ready(g));
    YK_TRY(stokes_lists(g));
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
    const int tpb = npp <= FAR_TPB ? 32 * ceil_div(npp, 32) : FAR_TPB;
    if (f32) {
        YK_LAUNCH(k_stokes_near32, np, tpb, sizeof(float4) * npp, st, npp, S.near_off,
                  S.near_idx, S.s32, g->d_xi, g->d_nx, g->d_ny, g->d_particles, -1.0 / S_PI, out);
        YK_LAUNCH(k_stokes_p2m<float>, np, 128, 0, st, npp, SP, S.s64, S.s32, g->d_particles,
                  (cx<float>*)S.coef32);
        YK_LAUNCH(k_stokes_m2l<float>, np, 256, 0, st, S.far_off, S.far,
                  (const cx<float>*)S.coef32, (cx<float>*)S.loc32, S.lmax32);
        YK_LAUNCH((k_stokes_l2p<float, 0>), np, 128, 0, st, npp, g->d_x, g->d_y, g->d_xi,
                  g->d_nx, g->d_ny, g->d_particles, (const cx<float>*)S.loc32, S.lmax32,
                  g->prm.viscosity, out);
        YK_TRY_CUDA(cudaGetLastError());
        return YK_OK;
    }
    const bool vel = which == STOKES_VELOCITY;
    if (vel)
        YK_LAUNCH(k_stokes_near64<1>, np, tpb, sizeof(double4) * npp, st, npp, S.near_off,
                  S.near_idx, S.s64, g->d_x, g->d_y, g->d_nx, g->d_ny,
                  1.0 / (4.0 * S_PI * g->prm.viscosity), out);
    else
        YK_LAUNCH(k_stokes_near64<0>, np, tpb, sizeof(double4) * npp, st, npp, S.near_off,
                  S.near_idx, S.s64, g->d_x, g->d_y, g->d_nx, g->d_ny, -1.0 / S_PI, out);
    YK_LAUNCH(k_stokes_p2m<double>, np, 128, 0, st, npp, SP, S.s64, S.s32, g->d_particles,
              (cx<double>*)S.coef64);
    YK_LAUNCH(k_stokes_m2l<double>, np, 256, 0, st, S.far_off, S.far,
              (const cx<double>*)S.coef64, (cx<double>*)S.loc64, S.lmax64);
    if (vel)
        YK_LAUNCH((k_stokes_l2p<double, 1>), np, 128, 0, st, npp, g->d_x, g->d_y, g->d_xi,
                  g->d_nx, g->d_ny, g->d_particles, (const cx<double>*)S.loc64, S.lmax64,
                  g->prm.viscosity, out);
    else
        YK_LAUNCH((k_stokes_l2p<double, 0>), np, 128, 0, st, npp, g->d_x, g->d_y, g->d_xi,
                  g->d_nx, g->d_ny, g->d_particles, (const cx<double>*)S.loc64, S.lmax64,
                  g->prm.viscosity, out);
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
