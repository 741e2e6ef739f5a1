// Discretisation (composite Gauss-Legendre panels, Section 6.2 / Table 1
// set-up), Dirichlet data (Eq. JanusBC and variants) and the QBX near-field
// rows (Section 5, Eqs. local-exp, graf-coefficient, graf-addition in their
// Yukawa form) of the screened-Laplace double layer.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "bessel.cuh"
#include "block_apply.cuh"
#include "yk_internal.cuh"

namespace yk {

// ---------------------------------------------------------------------------
// Gauss-Legendre rule on [-1, 1]: Newton's method on P_n (three-term
// recurrence) from the standard cosine initial guess; nodes ascending.
// ---------------------------------------------------------------------------
__global__ void k_gauss_legendre(int n, double* x, double* w) {
    int i = threadIdx.x;
    if (i >= n) return;
    int r = n - 1 - i;  // root index counted from the right end
    double t = cos(PI * (r + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        // P_n = p1, P_{n-1} = p0; P_n' = n (t P_n - P_{n-1}) / (t^2 - 1)
        dp = n * (t * p1 - p0) / (t * t - 1.0);
        double dt = p1 / dp;
        t -= dt;
        if (fabs(dt) < 1e-16) break;
    }
    {
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (t * p1 - p0) / (t * t - 1.0);
    }
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
}

// Reference-interval matrices: fine sub-panel nodes/weights, Lagrange
// interpolation (coarse GL nodes -> fine nodes) and differentiation at the
// GL nodes, both in barycentric form.
__global__ void k_ref_matrices(int ngl, int os, const double* glx, const double* glw,
                               double* fine_x, double* fine_w, double* interp, double* diff) {
    __shared__ double bw[MAX_NGL];
    int tid = threadIdx.x;
    if (tid < ngl) {
        double p = 1.0;
        for (int k = 0; k < ngl; ++k)
            if (k != tid) p *= (glx[tid] - glx[k]);
        bw[tid] = 1.0 / p;
    }
    __syncthreads();
    int nf = os * ngl;
    for (int f = tid; f < nf; f += blockDim.x) {
        int m = f / ngl, l = f % ngl;
        double xf = -1.0 + (2.0 / os) * (m + 0.5 * (glx[l] + 1.0));
        fine_x[f] = xf;
        fine_w[f] = glw[l] / os;
        // barycentric interpolation weights at xf
        int hit = -1;
        for (int j = 0; j < ngl; ++j)
            if (xf == glx[j]) hit = j;
        if (hit >= 0) {
            for (int j = 0; j < ngl; ++j) interp[f * ngl + j] = (j == hit) ? 1.0 : 0.0;
        } else {
            double den = 0.0;
            for (int j = 0; j < ngl; ++j) den += bw[j] / (xf - glx[j]);
            for (int j = 0; j < ngl; ++j) interp[f * ngl + j] = bw[j] / (xf - glx[j]) / den;
        }
    }
    for (int e = tid; e < ngl * ngl; e += blockDim.x) {
        int i = e / ngl, j = e % ngl;
        if (i != j) {
            diff[e] = (bw[j] / bw[i]) / (glx[i] - glx[j]);
        }
    }
    __syncthreads();
    for (int i = tid; i < ngl; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < ngl; ++j)
            if (j != i) s += diff[i * ngl + j];
        diff[i * ngl + i] = -s;
    }
}

// Boundary point and derivative of particle p at parameter t (Section 2.1).
__device__ __forceinline__ void curve_point(double cx, double cy, double cphi, double sphi,
                                            double A, double B, double t, double& x,
                                            double& y, double& dx, double& dy) {
    double ct, st;
    sincos(t, &st, &ct);
    double u = A * ct, v = B * st, du = -A * st, dv = B * ct;
    x = cx + cphi * u - sphi * v;
    y = cy + sphi * u + cphi * v;
    dx = cphi * du - sphi * dv;
    dy = sphi * du + cphi * dv;
}

__global__ void k_nodes(int64_t n, int npan, int ngl, const yk_particle* parts,
                        const double* glx, const double* glw, double* X, double* Y,
                        double* NX, double* NY, double* W, double* S, float2* XI) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int npp = npan * ngl;
    int p = (int)(i / npp);
    int li = (int)(i % npp);
    int k = li / ngl, j = li % ngl;
    double dt = 2.0 * PI / npan;
    double t = k * dt + 0.5 * dt * (glx[j] + 1.0);
    yk_particle P = parts[p];
    double sp, cp;
    sincos(P.phi, &sp, &cp);
    double x, y, dx, dy;
    curve_point(P.cx, P.cy, cp, sp, P.A, P.B, t, x, y, dx, dy);
    double spd = sqrt(dx * dx + dy * dy);
    X[i] = x;
    Y[i] = y;
    NX[i] = dy / spd;   // normal out of the particle: tangent rotated clockwise
    NY[i] = -dx / spd;
    W[i] = glw[j] * 0.5 * dt * spd;
    S[i] = spd;
    XI[i] = make_float2((float)(x - P.cx), (float)(y - P.cy));
}

// Per particle: centre, bounding radius and perimeter (sum of weights).
__global__ void k_particle_info(int np, int npp, const yk_particle* parts, const double* W,
                                yk::d4* out, float4* c32, float* r32) {
    int p = blockIdx.x;
    double s = 0.0;
    for (int j = threadIdx.x; j < npp; j += blockDim.x) s += W[(int64_t)p * npp + j];
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        yk_particle P = parts[p];
        out[p] = make_d4(P.cx, P.cy, fmax(P.A, P.B), red[0]);
        const float hx = (float)P.cx, hy = (float)P.cy;
        c32[p] = make_float4(hx, hy, (float)(P.cx - (double)hx), (float)(P.cy - (double)hy));
        r32[p] = (float)fmax(P.A, P.B);
    }
}

// Dirichlet data; theta measured from the director (Eq. JanusBC text).
__global__ void k_label(int64_t n, int npp, const yk_particle* parts, const double* X,
                        const double* Y, int kind, double param, double* f) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    yk_particle P = parts[i / npp];
    double rx = X[i] - P.cx, ry = Y[i] - P.cy;
    double rn = sqrt(rx * rx + ry * ry);
    double sp, cp;
    sincos(P.phi, &sp, &cp);
    double cth = (rx * cp + ry * sp) / rn;
    double sth = (cp * ry - sp * rx) / rn;
    double v;
    if (kind == YK_LABEL_TANH) {
        v = 0.5 * (1.0 + tanh(param * cth));
    } else if (kind == YK_LABEL_SINP) {
        int e = (int)param;
        double pw = 1.0;
        for (int k = 0; k < e; ++k) pw *= sth;
        v = 1.0 - pw;
    } else {
        v = 0.5 * (1.0 + cth);
    }
    f[i] = v;
}

// ---------------------------------------------------------------------------
// QBX near rows (Section 5). For target x on its particle's panel k, the
// expansion centre is c = x + r nu, r = r_factor * h_k (exterior side). The
// density on the near panels is resampled on `os` sub-panels per panel; the
// Yukawa double-layer coefficients are
//   alpha_n = (1/2pi) sum_f w_f sigma_f [ (nu.e_s) K_n'(s/rho)/rho
//                                         - i n (nu.e_phi) K_n(s/rho)/s ] e^{-i n phi_f}
// and u(x) = sum_{|n|<=p} alpha_n I_n(r/rho) e^{i n theta_x}. With
// Delta = theta_x - phi_f this is, per fine node, the real weight
//   v_f = (w_f/2pi) [A_0 I_0 + 2 sum_{n>=1} I_n (A_n cos nDelta + n B_n sin nDelta)]
// with A_n = (nu.e_s) K_n'/rho, B_n = (nu.e_phi) K_n / s. The normal
// derivative (nu . grad = -d/dr at the target) replaces I_n by -I_n'(r/rho)/rho.
// The fine weights are folded back onto the coarse near nodes through the
// panel-wise Lagrange interpolation matrix. A rigid particle's rows do not
// depend on its position or orientation, so they are built once per shape
// on a canonical copy (centre 0, phi 0).
// ---------------------------------------------------------------------------
__global__ void k_qbx_rows(int npan, int ngl, int near_w, int n_near, int os, int order,
                           double r_factor, double rho, double eta, const double2* shape_ab,
                           const double* glx, const double* glw, const double* fine_x,
                           const double* fine_w, const double* interp, double* cval,
                           double* cgrad) {
    extern __shared__ double sm[];
    const int npp = npan * ngl;
    const int s = blockIdx.y;
    const int li = blockIdx.x;
    const int nfp = os * ngl;          // fine nodes per near panel
    const int nf = n_near * nfp;       // fine nodes per target
    double* vf = sm;                   // [nf]
    double* vg = sm + nf;              // [nf]
    __shared__ double In[MAX_ORDER + 2], beta[MAX_ORDER + 1], gam[MAX_ORDER + 1];
    __shared__ double sh_c[2], sh_theta;
    const double A = shape_ab[s].x, B = shape_ab[s].y;
    const double dt = 2.0 * PI / npan;
    const int k = li / ngl, j = li % ngl;

    if (threadIdx.x == 0) {
        double t = k * dt + 0.5 * dt * (glx[j] + 1.0);
        double x, y, dx, dy;
        curve_point(0.0, 0.0, 1.0, 0.0, A, B, t, x, y, dx, dy);
        double spd = sqrt(dx * dx + dy * dy);
        double nx = dy / spd, ny = -dx / spd;
        double h = 0.0;  // panel arclength = sum of the panel's node weights
        for (int m = 0; m < ngl; ++m) {
            double tm = k * dt + 0.5 * dt * (glx[m] + 1.0);
            double xm, ym, dxm, dym;
            curve_point(0.0, 0.0, 1.0, 0.0, A, B, tm, xm, ym, dxm, dym);
            h += glw[m] * 0.5 * dt * sqrt(dxm * dxm + dym * dym);
        }
        double r = r_factor * h;
        sh_c[0] = x + r * nx;
        sh_c[1] = y + r * ny;
        sh_theta = atan2(-ny, -nx);
        In[MAX_ORDER + 1] = r;  // stash r for the other threads
    }
    __syncthreads();
    const double r = In[MAX_ORDER + 1];
    __syncthreads();
    if (threadIdx.x <= order + 1) In[threadIdx.x] = bessel_i_series(threadIdx.x, r / rho);
    __syncthreads();
    if (threadIdx.x <= order) {
        int n = threadIdx.x;
        double ip = (n == 0) ? In[1] : 0.5 * (In[n - 1] + In[n + 1]);
        beta[n] = In[n];
        gam[n] = -ip / rho;
    }
    __syncthreads();
    const double cx = sh_c[0], cy = sh_c[1], thx = sh_theta;

    for (int f = threadIdx.x; f < nf; f += blockDim.x) {
        int q = f / nfp, m = f % nfp;
        int pk = (2 * near_w + 1 >= npan) ? q : ((k - near_w + q) % npan + npan) % npan;
        double t = pk * dt + 0.5 * dt * (fine_x[m] + 1.0);
        double yx, yy, dx, dy;
        curve_point(0.0, 0.0, 1.0, 0.0, A, B, t, yx, yy, dx, dy);
        double spd = sqrt(dx * dx + dy * dy);
        double nux = dy / spd, nuy = -dx / spd;
        double wf = 0.5 * dt * fine_w[m] * spd;
        double ex = yx - cx, ey = yy - cy;
        double sd = sqrt(ex * ex + ey * ey);
        double phi = atan2(ey, ex);
        double esx = ex / sd, esy = ey / sd;
        double a_s = nux * esx + nuy * esy;      // nu . e_s
        double a_p = -nux * esy + nuy * esx;     // nu . e_phi, e_phi = (-e_s.y, e_s.x)
        double z = sd / rho;
        double Kn[MAX_ORDER + 2];
        k01(z, Kn[0], Kn[1]);
        for (int n = 1; n <= order; ++n) Kn[n + 1] = Kn[n - 1] + (2.0 * n / z) * Kn[n];
        double dlt = thx - phi;
        double c1, s1;
        sincos(dlt, &s1, &c1);
        // n = 0 term: A_0 = a_s K_0'/rho = -a_s K_1 / rho; the single layer's
        // coefficient (combined representation) adds eta K_n(s/rho) e^{-in phi}
        double A0 = -a_s * Kn[1] / rho + eta * Kn[0];
        double v = beta[0] * A0, vn = gam[0] * A0;
        double cn = 1.0, sn = 0.0;
        for (int n = 1; n <= order; ++n) {
            double cn1 = cn * c1 - sn * s1;
            sn = sn * c1 + cn * s1;
            cn = cn1;
            double kp = -0.5 * (Kn[n - 1] + Kn[n + 1]);
            double An = a_s * kp / rho;
            double Bn = a_p * Kn[n] / sd;
            double term = An * cn + n * Bn * sn + eta * Kn[n] * cn;
            v += 2.0 * beta[n] * term;
            vn += 2.0 * gam[n] * term;
        }
        vf[f] = v * wf / (2.0 * PI);
        vg[f] = vn * wf / (2.0 * PI);
    }
    __syncthreads();
    const int rowlen = n_near * ngl;
    double* crow = cval + ((int64_t)s * npp + li) * rowlen;
    double* grow = cgrad + ((int64_t)s * npp + li) * rowlen;
    for (int c = threadIdx.x; c < rowlen; c += blockDim.x) {
        int q = c / ngl, jj = c % ngl;
        double av = 0.0, ag = 0.0;
        const double* vq = vf + q * nfp;
        const double* gq = vg + q * nfp;
        for (int m = 0; m < nfp; ++m) {
            double L = interp[m * ngl + jj];
            av = fma(vq[m], L, av);
            ag = fma(gq[m], L, ag);
        }
        crow[c] = av;
        grow[c] = ag;
    }
}

// ---------------------------------------------------------------------------
// Block preconditioner. The self-interaction block of a particle (targets
// and sources on the same particle: QBX rows for near columns, the plain
// double-layer kernel otherwise) depends only on its shape, so one block and
// its inverse serve every particle of that shape. GMRES is right
// preconditioned by blockdiag(inverse blocks).
// ---------------------------------------------------------------------------
__global__ void k_self_block(int npan, int ngl, int near_w, int n_near, double rho, double eta,
                             const double2* shape_ab, const double* glx, const double* glw,
                             const double* cval, double* A) {
    const int npp = npan * ngl;
    const int s = blockIdx.y, i = blockIdx.x;
    const double a = shape_ab[s].x, b = shape_ab[s].y;
    const double dt = 2.0 * PI / npan;
    const int k = i / ngl;
    double xi, yi, dxi, dyi;
    curve_point(0.0, 0.0, 1.0, 0.0, a, b, k * dt + 0.5 * dt * (glx[i % ngl] + 1.0), xi, yi, dxi,
                dyi);
    const int rowlen = n_near * ngl;
    const double* row = cval + ((int64_t)s * npp + i) * rowlen;
    double* out = A + ((int64_t)s * npp + i) * npp;
    const bool all_near = 2 * near_w + 1 >= npan;
    for (int j = threadIdx.x; j < npp; j += blockDim.x) {
        const int kj = j / ngl;
        int d = ((kj - k) % npan + npan) % npan;
        const bool near = all_near || d <= near_w || npan - d <= near_w;
        double v;
        if (near) {
            const int q = all_near ? kj : ((kj - k + near_w) % npan + npan) % npan;
            v = row[q * ngl + (j % ngl)];
        } else {
            double x, y, dx, dy;
            curve_point(0.0, 0.0, 1.0, 0.0, a, b, kj * dt + 0.5 * dt * (glx[j % ngl] + 1.0), x, y,
                        dx, dy);
            const double spd = sqrt(dx * dx + dy * dy);
            const double nx = dy / spd, ny = -dx / spd;
            const double w = glw[j % ngl] * 0.5 * dt * spd;
            const double ex = xi - x, ey = yi - y;
            const double r = sqrt(ex * ex + ey * ey);
            double k0v, k1v;
            k01(r / rho, k0v, k1v);
            v = (k1v * (ex * nx + ey * ny) / (rho * r) + eta * k0v) / (2.0 * PI) * w;
        }
        out[j] = v;
    }
}

// Inverse of the self block by the Newton-Schulz (hyperpower, order 2)
// iteration X <- X (2I - A X) (G. Schulz, ZAMM 13, 1933), in FP32. The
// inverse only preconditions GMRES: it is applied as a fixed linear operator,
// so its rounding changes the convergence rate, not the solution. Starting
// from X0 = A^T / (|A|_1 |A|_inf), every singular value of A X0 lies in
// (0, 1], and each step maps s -> s (2 - s): small singular values double
// until they near 1, then the residual I - A X squares. The block (1/2 I plus
// a compact part) is well conditioned, so this takes about ten steps, each two
// batched n x n GEMMs spread over many SMs.

// Column and row sums of |A| (FP64 block -> FP32 copy), one CTA per shape:
// scale[s] = 1 / (max column sum * max row sum).
__global__ void k_ns_setup(int n, const double* __restrict__ A, float* __restrict__ A32,
                           float* __restrict__ scale) {
    const int s = blockIdx.x;
    const double* As = A + (int64_t)s * n * n;
    float* Bs = A32 + (int64_t)s * n * n;
    double cmax = 0.0, rmax = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double c = 0.0, r = 0.0;
        for (int i = 0; i < n; ++i) {
            c += fabs(As[(int64_t)i * n + j]);
            r += fabs(As[(int64_t)j * n + i]);
        }
        cmax = fmax(cmax, c);
        rmax = fmax(rmax, r);
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) Bs[e] = (float)As[e];
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    }
    if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = cmax, red[1][threadIdx.x >> 5] = rmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double c = 0.0, r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) c = fmax(c, red[0][w]), r = fmax(r, red[1][w]);
        scale[s] = (float)(1.0 / (c * r));
    }
}

// X0 = scale * A^T (FP32).
__global__ void k_ns_init(int n, const float* __restrict__ A32, const float* __restrict__ scale,
                          float* __restrict__ X) {
    const int s = blockIdx.y;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int i = (int)(e / n), j = (int)(e % n);
    X[(int64_t)s * n * n + e] = scale[s] * A32[(int64_t)s * n * n + (int64_t)j * n + i];
}

// Batched C_s = L_s R_s for n x n row-major FP32 matrices (blockIdx.z = s),
// 64 x 64 output tile per CTA, 16-deep k slices staged in shared memory, each
// of 256 threads accumulating a 4 x 4 block (rows ty + 16a, columns tx + 16b).
// RESID: the product is T = A X; the epilogue stores 2I - T and raises
// *err_bits to the largest |(I - T)_ij| (non-negative floats order like their
// bit patterns).
constexpr int NS_TILE = 64, NS_K = 16;
template <bool RESID>
__global__ void __launch_bounds__(256) k_ns_gemm(int n, const float* __restrict__ L,
                                                 const float* __restrict__ R,
                                                 float* __restrict__ C,
                                                 unsigned* __restrict__ err_bits) {
    __shared__ float Ls[NS_K][NS_TILE + 4];
    __shared__ float Rs[NS_K][NS_TILE + 4];
    const int64_t off = (int64_t)blockIdx.z * n * n;
    L += off;
    R += off;
    C += off;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = blockIdx.y * NS_TILE, col0 = blockIdx.x * NS_TILE;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
    for (int k0 = 0; k0 < n; k0 += NS_K) {
        for (int e = threadIdx.x; e < NS_TILE * NS_K; e += 256) {
            const int r = e / NS_K, k = e % NS_K;
            const int gr = row0 + r, gk = k0 + k;
            Ls[k][r] = (gr < n && gk < n) ? L[(int64_t)gr * n + gk] : 0.0f;
            const int kk = e / NS_TILE, c = e % NS_TILE;
            const int gk2 = k0 + kk, gc = col0 + c;
            Rs[kk][c] = (gk2 < n && gc < n) ? R[(int64_t)gk2 * n + gc] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NS_K; ++k) {
            float l[4], r[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) l[a] = Ls[k][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) r[b] = Rs[k][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(l[a], r[b], acc[a][b]);
        }
        __syncthreads();
    }
    float emax = 0.0f;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = row0 + ty + 16 * a, j = col0 + tx + 16 * b;
            if (i < n && j < n) {
                float v = acc[a][b];
                if (RESID) {
                    const float res = (i == j ? 1.0f : 0.0f) - v;
                    emax = fmaxf(emax, fabsf(res));
                    v = (i == j ? 1.0f : 0.0f) + res;
                }
                C[(int64_t)i * n + j] = v;
            }
        }
    if (RESID) {
        for (int o = 16; o > 0; o >>= 1) emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        if ((threadIdx.x & 31) == 0) atomicMax(err_bits, __float_as_uint(emax));
    }
}

// minv[s][j][i] = X[s][i][j] in FP64 and FP32.
__global__ void k_ns_store(int n, const float* __restrict__ X, double* __restrict__ minv,
                           float* __restrict__ minv32) {
    const int s = blockIdx.y;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int j = (int)(e / n), i = (int)(e % n);
    const float v = X[(int64_t)s * n * n + (int64_t)i * n + j];
    minv[(int64_t)s * n * n + e] = (double)v;
    minv32[(int64_t)s * n * n + e] = v;
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// Far part of the self-interaction block of each shape: own-particle sources
// outside the target's near panels (zero on the near columns, which the QBX
// rows cover), for the value (GRAD = false: dG/dnu_y, Eq. double-layer-def)
// or the normal derivative (GRAD = true: nu_x . grad_x dG/dnu_y), quadrature
// weights included, stored transposed (S[s][j][i]). Both depend only on the
// shape: the kernels involve only distances and dot products of normals,
// which rigid motions keep, so the blocks are built once in the particle frame.
template <bool GRAD>
__global__ void k_self_far(int npan, int ngl, int near_w, double rho, double eta,
                           const double2* shape_ab,
                           const double* glx, const double* glw, double* S) {
    const int npp = npan * ngl;
    const int s = blockIdx.y, i = blockIdx.x;
    const double a = shape_ab[s].x, b = shape_ab[s].y;
    const double dt = 2.0 * PI / npan;
    const int k = i / ngl;
    double xi, yi, dxi, dyi;
    curve_point(0.0, 0.0, 1.0, 0.0, a, b, k * dt + 0.5 * dt * (glx[i % ngl] + 1.0), xi, yi, dxi,
                dyi);
    const double spi = sqrt(dxi * dxi + dyi * dyi);
    const double nxi = dyi / spi, nyi = -dxi / spi;
    double* out = S + (int64_t)s * npp * npp;
    const bool all_near = 2 * near_w + 1 >= npan;
    for (int j = threadIdx.x; j < npp; j += blockDim.x) {
        const int kj = j / ngl;
        const int d = ((kj - k) % npan + npan) % npan;
        double v = 0.0;
        if (!(all_near || d <= near_w || npan - d <= near_w)) {
            double x, y, dx, dy;
            curve_point(0.0, 0.0, 1.0, 0.0, a, b, kj * dt + 0.5 * dt * (glx[j % ngl] + 1.0), x, y,
                        dx, dy);
            const double spd = sqrt(dx * dx + dy * dy);
            const double nx = dy / spd, ny = -dx / spd;
            const double w = glw[j % ngl] * 0.5 * dt * spd;
            const double ex = xi - x, ey = yi - y;
            const double r = sqrt(ex * ex + ey * ey);
            double k0v, k1v;
            k01(r / rho, k0v, k1v);
            const double dn_s = ex * nx + ey * ny;
            if (!GRAD) {
                v = (k1v * dn_s / (rho * r) + eta * k0v) / (2.0 * PI) * w;
            } else {
                const double gg = k1v / (r * rho);
                const double gp = -(k0v / rho + 2.0 * k1v / r) / (rho * r);
                const double nn = nxi * nx + nyi * ny;
                const double dn_t = ex * nxi + ey * nyi;
                // + eta nu_x . grad_x G = -eta K1(r/rho) (d . nu_x) / (rho r)
                v = (gg * nn + gp * dn_s * dn_t / r - eta * k1v * dn_t / (rho * r)) * w /
                    (2.0 * PI);
            }
        }
        out[(int64_t)j * npp + i] = v;
    }
}

// Newton-Schulz steps: stop once the largest entry of I - A X is below
// NS_TOL, or once it is below 1e-3 and has stopped shrinking (the FP32
// floor). A block whose residual does not fall below 1/2 is singular to
// working precision.
constexpr int NS_MAX_STEPS = 100;
constexpr float NS_TOL = 1e-6f;

int build_preconditioner(yk_geom* g) {
    if (g->prm.precond != YK_PRECOND_BLOCK) return YK_OK;
    cudaStream_t st = g->ctx->stream;
    double* hs = host_status(g->ctx);
    if (!hs) return YK_ERR_NO_MEMORY;
    const int n = g->npp, ns = g->nshape;
    const size_t nn = (size_t)n * n;
    double* A = nullptr;
    float* W = nullptr;
    YK_TRY(dev_alloc((void**)&A, sizeof(double) * nn * ns, st));
    int rc = dev_alloc((void**)&W, sizeof(float) * (4 * nn * ns + ns + 32), st);
    if (rc != YK_OK) {
        dev_free(A, st);
        return rc;
    }
    float* A32 = W;
    float* X = W + nn * ns;
    float* T = W + 2 * nn * ns;
    float* Xn = W + 3 * nn * ns;
    float* scale = W + 4 * nn * ns;
    unsigned* err_bits = reinterpret_cast<unsigned*>(scale + ns);
    YK_LAUNCH(k_self_block, dim3(n, ns), 128, 0, st, g->npan, g->ngl, g->prm.near_width,
              g->n_near, g->prm.rho, g->view().eta, g->d_shape_ab, g->d_glx, g->d_glw, g->d_cval,
              A);
    YK_LAUNCH(k_ns_setup, ns, 256, 0, st, n, A, A32, scale);
    const dim3 eg((unsigned)((nn + 255) / 256), ns);
    YK_LAUNCH(k_ns_init, eg, 256, 0, st, n, A32, scale, X);
    const dim3 gg((n + NS_TILE - 1) / NS_TILE, (n + NS_TILE - 1) / NS_TILE, ns);
    float prev = INFINITY, err = INFINITY;
    for (int it = 0; it < NS_MAX_STEPS; ++it) {
        // T = 2I - A X, recording max |I - A X|; then X <- X T
        if (cudaMemsetAsync(err_bits, 0, sizeof(unsigned), st) != cudaSuccess) {
            rc = YK_ERR_CUDA;
            break;
        }
        YK_LAUNCH(k_ns_gemm<true>, gg, 256, 0, st, n, A32, X, T, err_bits);
        unsigned bits = 0;
        if (cudaMemcpyAsync(hs, err_bits, sizeof(unsigned), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = YK_ERR_CUDA;
            break;
        }
        std::memcpy(&bits, hs, sizeof(unsigned));
        std::memcpy(&err, &bits, sizeof(float));
        if (!(err == err)) break;                                   // NaN: singular
        if (err < NS_TOL || (err < 1e-3f && err > 0.25f * prev)) break;
        YK_LAUNCH(k_ns_gemm<false>, gg, 256, 0, st, n, X, T, Xn, nullptr);
        std::swap(X, Xn);
        prev = err;
    }
    if (rc == YK_OK && !(err < 0.5f)) rc = YK_ERR_BAD_GEOMETRY;
    if (rc == YK_OK) {
        YK_LAUNCH(k_ns_store, eg, 256, 0, st, n, X, g->d_minv, g->d_minv32);
        if (cudaGetLastError() != cudaSuccess) rc = YK_ERR_CUDA;
    }
    dev_free(A, st);
    dev_free(W, st);
    return rc;
}

int apply_preconditioner(yk_geom* g, const double* x, double* y, bool fp32) {
    cudaStream_t st = g->ctx->stream;
    // y_P = inv(block of P's shape) x_P
    const dim3 grid(g->np, ceil_div(g->npp, BAPPLY_ROWS));
    if (fp32)
        YK_LAUNCH((k_blocks_apply<float, false>), grid, BAPPLY_ROWS * BAPPLY_SLICES,
                  blocks_apply_smem<float>(g->npp), st, g->npp, g->d_shape_of, g->d_minv32, x, y);
    else
        YK_LAUNCH((k_blocks_apply<double, false>), grid, BAPPLY_ROWS * BAPPLY_SLICES,
                  blocks_apply_smem<double>(g->npp), st, g->npp, g->d_shape_of, g->d_minv, x, y);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

// Node arrays and per-particle data from the current particle list.
int update_nodes(yk_geom* g) {
    cudaStream_t st = g->ctx->stream;
    yk_particle* d_parts = g->d_particles;   // the geometry's device copy of the particles
    YK_TRY_CUDA(cudaMemcpyAsync(d_parts, g->parts.data(), sizeof(yk_particle) * g->np,
                                cudaMemcpyHostToDevice, st));
    YK_LAUNCH(k_nodes, ceil_div(g->n, 256), 256, 0, st, g->n, g->npan, g->ngl, d_parts, g->d_glx,
              g->d_glw, g->d_x, g->d_y, g->d_nx, g->d_ny, g->d_w, g->d_speed, g->d_xi);
    YK_LAUNCH(k_particle_info, g->np, 256, 0, st, g->np, g->npp, d_parts, g->d_w, g->d_part,
              g->d_c32, g->d_r32);
    for (auto& L : g->lists) L.valid = false;   // particle pairs change when particles move
    for (auto& L : g->sym) L.valid = false;
    g->nbr_valid = false;
    g->fmm.valid = false;                       // the quadtree follows the particles
    for (auto& B : g->bands) B.valid = false;
    g->contact.valid = false;                   // so do the near-contact lists
    g->stokes.lists_valid = false;              // and the Stokes pair lists
    g->coarse.valid = false;                    // and the coarse space's couplings
    YK_TRY_CUDA(cudaGetLastError());
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    return YK_OK;
}

// ---------------------------------------------------------------------------
// Per-shape precomputation shared across geometries. A rigid shape's QBX
// rows (value and normal derivative), its self blocks and the inverse of its
// self-interaction block depend on the shape, the discretisation and rho,
// not on where the particle sits or how it is turned. A process-wide cache,
// per device, keeps them keyed by every parameter they depend on, so that a
// geometry whose shapes were seen before (the same shapes solved again, a
// stream of requests drawn from a few shapes) copies them instead of forming
// the QBX coefficients and running the Newton-Schulz inversion again. The
// first geometry of a shape computes and inserts it. Entries are device
// buffers of their own (cudaMalloc), evicted least recently used beyond
// SHAPE_CACHE_BYTES; they live until evicted or the process exits.
// ---------------------------------------------------------------------------
constexpr size_t SHAPE_CACHE_BYTES = (size_t)4 << 30;

struct ShapeKey {
    int device, npan, ngl, near_w, os, order, precond, use_self;
    double A, B, r_factor, rho, eta;
    bool operator<(const ShapeKey& o) const {
        return std::tie(device, npan, ngl, near_w, os, order, precond, use_self, A, B, r_factor,
                        rho, eta) < std::tie(o.device, o.npan, o.ngl, o.near_w, o.os, o.order,
                                             o.precond, o.use_self, o.A, o.B, o.r_factor, o.rho,
                                             o.eta);
    }
};

struct ShapeEntry {
    void* buf = nullptr;     // rows (cval, cgrad), blocks (self, self_grad, minv), FP32 blocks
    size_t bytes = 0;
    uint64_t last_use = 0;
};

static std::mutex g_shape_mutex;
static std::map<ShapeKey, ShapeEntry> g_shape_cache;
static size_t g_shape_bytes = 0;
static uint64_t g_shape_clock = 0;

// Byte offsets of one shape's arrays inside an entry's buffer.
struct ShapeLayout {
    size_t rows, blk, cval, cgrad, self, self_grad, minv, self32, minv32, total;
    explicit ShapeLayout(const yk_geom* g) {
        const bool has_self = g->use_self, has_pc = g->prm.precond == YK_PRECOND_BLOCK;
        rows = (size_t)g->npp * g->n_near * g->ngl * sizeof(double);
        blk = (size_t)g->npp * g->npp;
        cval = 0;
        cgrad = cval + rows;
        self = cgrad + rows;
        self_grad = self + (has_self ? blk * sizeof(double) : 0);
        minv = self_grad + (has_self ? blk * sizeof(double) : 0);
        self32 = minv + (has_pc ? blk * sizeof(double) : 0);
        minv32 = self32 + (has_self ? blk * sizeof(float) : 0);
        total = minv32 + (has_pc ? blk * sizeof(float) : 0);
    }
};

static ShapeKey shape_key(const yk_geom* g, int s) {
    ShapeKey k;
    k.device = g->ctx->device;
    k.npan = g->npan;
    k.ngl = g->ngl;
    k.near_w = g->prm.near_width;
    k.os = g->prm.oversample;
    k.order = g->prm.qbx_order;
    k.precond = g->prm.precond;
    k.use_self = g->use_self ? 1 : 0;
    k.A = g->shape_ab[s].x;
    k.B = g->shape_ab[s].y;
    k.r_factor = g->prm.qbx_r_factor;
    k.rho = g->prm.rho;
    k.eta = g->view().eta;
    return k;
}

// Copy shape s's arrays between the geometry and a cache buffer (to_cache:
// geometry -> buffer), on the geometry's stream.
static int shape_copy(yk_geom* g, int s, char* buf, bool to_cache) {
    const ShapeLayout L(g);
    cudaStream_t st = g->ctx->stream;
    const size_t rs = L.rows / sizeof(double), bs = L.blk;
    struct Part {
        void* geom;
        size_t off, bytes;
    } parts[] = {
        {g->d_cval + s * rs, L.cval, L.rows},
        {g->d_cgrad + s * rs, L.cgrad, L.rows},
        {g->use_self ? (void*)(g->d_self + s * bs) : nullptr, L.self, bs * sizeof(double)},
        {g->use_self ? (void*)(g->d_self_grad + s * bs) : nullptr, L.self_grad, bs * sizeof(double)},
        {g->d_minv ? (void*)(g->d_minv + s * bs) : nullptr, L.minv, bs * sizeof(double)},
        {g->use_self ? (void*)(g->d_self32 + s * bs) : nullptr, L.self32, bs * sizeof(float)},
        {g->d_minv32 ? (void*)(g->d_minv32 + s * bs) : nullptr, L.minv32, bs * sizeof(float)},
    };
    for (const Part& p : parts) {
        if (!p.geom) continue;
        void* dst = to_cache ? (void*)(buf + p.off) : p.geom;
        const void* src = to_cache ? (const void*)p.geom : (const void*)(buf + p.off);
        YK_TRY_CUDA(cudaMemcpyAsync(dst, src, p.bytes, cudaMemcpyDeviceToDevice, st));
    }
    return YK_OK;
}

// Fill every shape's arrays from the cache; true if all shapes were there.
static bool shapes_from_cache(yk_geom* g) {
    std::lock_guard<std::mutex> lk(g_shape_mutex);
    std::vector<ShapeEntry*> hit;
    for (int s = 0; s < g->nshape; ++s) {
        auto it = g_shape_cache.find(shape_key(g, s));
        if (it == g_shape_cache.end()) return false;
        hit.push_back(&it->second);
    }
    for (int s = 0; s < g->nshape; ++s) {
        hit[s]->last_use = ++g_shape_clock;
        if (shape_copy(g, s, (char*)hit[s]->buf, false) != YK_OK) return false;
    }
    // the copies are stream-ordered; an entry is freed only after a device
    // synchronisation (cudaFree), so it outlives them
    return true;
}

static void shapes_to_cache(yk_geom* g) {
    const ShapeLayout L(g);
    std::lock_guard<std::mutex> lk(g_shape_mutex);
    for (int s = 0; s < g->nshape; ++s) {
        const ShapeKey k = shape_key(g, s);
        if (g_shape_cache.count(k)) continue;
        while (g_shape_bytes + L.total > SHAPE_CACHE_BYTES && !g_shape_cache.empty()) {
            auto lru = g_shape_cache.begin();
            for (auto it = g_shape_cache.begin(); it != g_shape_cache.end(); ++it)
                if (it->second.last_use < lru->second.last_use) lru = it;
            cudaFree(lru->second.buf);   // synchronises the device: no copy from it is pending
            g_shape_bytes -= lru->second.bytes;
            g_shape_cache.erase(lru);
        }
        if (L.total > SHAPE_CACHE_BYTES) return;
        ShapeEntry e;
        if (cudaMalloc(&e.buf, L.total) != cudaSuccess) {
            cudaGetLastError();
            return;   // no room: the geometry keeps its own copy, nothing is cached
        }
        if (shape_copy(g, s, (char*)e.buf, true) != YK_OK) {
            cudaFree(e.buf);
            return;
        }
        e.bytes = L.total;
        e.last_use = ++g_shape_clock;
        g_shape_bytes += e.bytes;
        g_shape_cache[k] = e;
    }
}

int build_geometry(yk_geom* g) {
    cudaStream_t st = g->ctx->stream;
    const yk_params& P = g->prm;
    const int os = P.oversample;
    YK_LAUNCH(k_gauss_legendre, 1, 32, 0, st, g->ngl, g->d_glx, g->d_glw);
    YK_LAUNCH(k_ref_matrices, 1, 256, 0, st, g->ngl, os, g->d_glx, g->d_glw, g->d_fine_x,
              g->d_fine_w, g->d_interp, g->d_diff);
    YK_TRY(update_nodes(g));
    if (shapes_from_cache(g)) {
        YK_TRY_CUDA(cudaGetLastError());
        YK_TRY_CUDA(cudaStreamSynchronize(st));
        return YK_OK;
    }
    const int nf = g->n_near * os * g->ngl;
    const size_t smem = 2 * sizeof(double) * nf;
    if (smem > 48 * 1024)
        YK_TRY_CUDA(cudaFuncSetAttribute(k_qbx_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    dim3 grid(g->npp, g->nshape);
    YK_LAUNCH(k_qbx_rows, grid, 128, smem, st, g->npan, g->ngl, P.near_width, g->n_near, os,
              P.qbx_order, P.qbx_r_factor, P.rho, g->view().eta, g->d_shape_ab, g->d_glx, g->d_glw,
              g->d_fine_x, g->d_fine_w, g->d_interp, g->d_cval, g->d_cgrad);
    if (g->use_self) {
        YK_LAUNCH(k_self_far<false>, grid, 128, 0, st, g->npan, g->ngl, P.near_width, P.rho,
                  g->view().eta, g->d_shape_ab, g->d_glx, g->d_glw, g->d_self);
        YK_LAUNCH(k_self_far<true>, grid, 128, 0, st, g->npan, g->ngl, P.near_width, P.rho,
                  g->view().eta, g->d_shape_ab, g->d_glx, g->d_glw, g->d_self_grad);
        const int64_t cnt = (int64_t)g->nshape * g->npp * g->npp;
        YK_LAUNCH(k_to_f32, ceil_div(cnt, 256), 256, 0, st, cnt, g->d_self, g->d_self32);
    }
    YK_TRY_CUDA(cudaGetLastError());
    YK_TRY(build_preconditioner(g));
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    shapes_to_cache(g);
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    return YK_OK;
}

int launch_label(yk_geom* g, int kind, double param, double* f) {
    cudaStream_t st = g->ctx->stream;
    yk_particle* d_parts = nullptr;
    YK_TRY(dev_alloc((void**)&d_parts, sizeof(yk_particle) * g->np, st));
    YK_TRY_CUDA(cudaMemcpyAsync(d_parts, g->parts.data(), sizeof(yk_particle) * g->np,
                                cudaMemcpyHostToDevice, st));
    YK_LAUNCH(k_label, ceil_div(g->n, 256), 256, 0, st, g->n, g->npp, d_parts, g->d_x, g->d_y, kind,
                                                 param, f);
    YK_TRY_CUDA(cudaGetLastError());
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    dev_free(d_parts, st);
    return YK_OK;
}

}  // namespace yk
