// Discretisation (composite Gauss-Legendre panels, Section 6.2 / Table 1
// set-up), Dirichlet data (Eq. JanusBC and variants) and the QBX near-field
// rows (Section 5, Eqs. local-exp, graf-coefficient, graf-addition in their
// Yukawa form) of the screened-Laplace double layer.
#include <math.h>

#include <algorithm>

#include "bessel.cuh"
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
                           double r_factor, double rho, const double2* shape_ab,
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
        // n = 0 term: A_0 = a_s K_0'/rho = -a_s K_1 / rho
        double A0 = -a_s * Kn[1] / rho;
        double v = beta[0] * A0, vn = gam[0] * A0;
        double cn = 1.0, sn = 0.0;
        for (int n = 1; n <= order; ++n) {
            double cn1 = cn * c1 - sn * s1;
            sn = sn * c1 + cn * s1;
            cn = cn1;
            double kp = -0.5 * (Kn[n - 1] + Kn[n + 1]);
            double An = a_s * kp / rho;
            double Bn = a_p * Kn[n] / sd;
            double term = An * cn + n * Bn * sn;
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
__global__ void k_self_block(int npan, int ngl, int near_w, int n_near, double rho,
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
            v = k1v * (ex * nx + ey * ny) / (2.0 * PI * rho * r) * w;
        }
        out[j] = v;
    }
}

// In-place Gauss-Jordan inversion with partial pivoting of the n x n block
// of shape blockIdx.x, on the augmented n x 2n matrix W (one CTA per shape),
// in FP32: the inverse only preconditions GMRES (it is applied as a fixed
// linear operator, so its own rounding changes the convergence rate, not the
// solution), and the block (1/2 I plus a compact part) is well conditioned.
// Writes the inverse transposed (minv[j][i] = inv[i][j]) in FP64 and FP32.
__global__ void __launch_bounds__(1024) k_gauss_jordan(int n, const double* A, float* W,
                                                       double* minv, float* minv32) {
    const int s = blockIdx.x;
    const double* As = A + (int64_t)s * n * n;
    float* Ws = W + (int64_t)s * n * 2 * n;
    const int n2 = 2 * n;
    extern __shared__ float fac[];             // n factors
    __shared__ float red_v[32];
    __shared__ int red_i[32];
    __shared__ int piv_row;
    for (int e = threadIdx.x; e < n * n2; e += blockDim.x) {
        const int r = e / n2, c = e % n2;
        Ws[e] = (c < n) ? (float)As[(int64_t)r * n + c] : (c - n == r ? 1.0f : 0.0f);
    }
    __syncthreads();
    for (int c = 0; c < n; ++c) {
        // pivot: row r >= c with the largest |W[r][c]|
        float best = -1.0f;
        int bi = c;
        for (int r = c + threadIdx.x; r < n; r += blockDim.x) {
            const float v = fabsf(Ws[(int64_t)r * n2 + c]);
            if (v > best) best = v, bi = r;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
        }
        if ((threadIdx.x & 31) == 0) red_v[threadIdx.x >> 5] = best, red_i[threadIdx.x >> 5] = bi;
        __syncthreads();
        if (threadIdx.x == 0) {
            float bv = -1.0f;
            int b = c;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (red_v[w] > bv) bv = red_v[w], b = red_i[w];
            piv_row = b;
        }
        __syncthreads();
        const int pr = piv_row;
        if (pr != c)
            for (int col = threadIdx.x; col < n2; col += blockDim.x) {
                const float t = Ws[(int64_t)c * n2 + col];
                Ws[(int64_t)c * n2 + col] = Ws[(int64_t)pr * n2 + col];
                Ws[(int64_t)pr * n2 + col] = t;
            }
        __syncthreads();
        const float inv_p = 1.0f / Ws[(int64_t)c * n2 + c];
        __syncthreads();
        for (int col = threadIdx.x; col < n2; col += blockDim.x) Ws[(int64_t)c * n2 + col] *= inv_p;
        for (int r = threadIdx.x; r < n; r += blockDim.x) fac[r] = (r == c) ? 0.0f : Ws[(int64_t)r * n2 + c];
        __syncthreads();
        for (int e = threadIdx.x; e < n * n2; e += blockDim.x) {
            const int r = e / n2, col = e % n2;
            const float f = fac[r];
            if (f != 0.0f) Ws[e] = fmaf(-f, Ws[(int64_t)c * n2 + col], Ws[e]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        const float v = Ws[(int64_t)i * n2 + n + j];
        minv[(int64_t)s * n * n + (int64_t)j * n + i] = (double)v;
        minv32[(int64_t)s * n * n + (int64_t)j * n + i] = v;
    }
}

// y_P = inv(block of P's shape) x_P, one CTA per particle.
template <typename T>
__global__ void k_block_apply(int np, int npp, const int* __restrict__ shape_of,
                              const T* __restrict__ minv, const double* __restrict__ x,
                              double* __restrict__ y) {
    extern __shared__ unsigned char smraw[];
    T* xs = reinterpret_cast<T*>(smraw);
    const int p = blockIdx.x;
    const int64_t base = (int64_t)p * npp;
    for (int j = threadIdx.x; j < npp; j += blockDim.x) xs[j] = (T)x[base + j];
    __syncthreads();
    const T* M = minv + (int64_t)shape_of[p] * npp * npp;
    for (int i = threadIdx.x; i < npp; i += blockDim.x) {
        T acc = 0;
        for (int j = 0; j < npp; ++j) acc += M[(int64_t)j * npp + i] * xs[j];
        y[base + i] = (double)acc;
    }
}

int build_preconditioner(yk_geom* g) {
    if (g->prm.precond != YK_PRECOND_BLOCK) return YK_OK;
    cudaStream_t st = g->ctx->stream;
    const int npp = g->npp;
    const size_t nn = (size_t)npp * npp;
    double* A = nullptr;
    float* W = nullptr;
    YK_TRY(dev_alloc((void**)&A, sizeof(double) * nn * g->nshape, st));
    YK_TRY(dev_alloc((void**)&W, sizeof(float) * 2 * nn * g->nshape, st));
    dim3 grid(npp, g->nshape);
    YK_LAUNCH(k_self_block, grid, 128, 0, st, g->npan, g->ngl, g->prm.near_width, g->n_near,
              g->prm.rho, g->d_shape_ab, g->d_glx, g->d_glw, g->d_cval, A);
    YK_LAUNCH(k_gauss_jordan, g->nshape, 1024, sizeof(float) * npp, st, npp, A, W, g->d_minv,
              g->d_minv32);
    YK_TRY_CUDA(cudaGetLastError());
    dev_free(A, st);
    dev_free(W, st);
    return YK_OK;
}

int apply_preconditioner(yk_geom* g, const double* x, double* y, bool fp32) {
    cudaStream_t st = g->ctx->stream;
    if (fp32)
        YK_LAUNCH(k_block_apply<float>, g->np, 256, sizeof(float) * g->npp, st, g->np, g->npp,
                  g->d_shape_of, g->d_minv32, x, y);
    else
        YK_LAUNCH(k_block_apply<double>, g->np, 256, sizeof(double) * g->npp, st, g->np, g->npp,
                  g->d_shape_of, g->d_minv, x, y);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

// Node arrays and per-particle data from the current particle list.
int update_nodes(yk_geom* g) {
    cudaStream_t st = g->ctx->stream;
    yk_particle* d_parts = nullptr;
    YK_TRY(dev_alloc((void**)&d_parts, sizeof(yk_particle) * g->np, st));
    YK_TRY_CUDA(cudaMemcpyAsync(d_parts, g->parts.data(), sizeof(yk_particle) * g->np,
                                cudaMemcpyHostToDevice, st));
    YK_LAUNCH(k_nodes, ceil_div(g->n, 256), 256, 0, st, g->n, g->npan, g->ngl, d_parts, g->d_glx,
              g->d_glw, g->d_x, g->d_y, g->d_nx, g->d_ny, g->d_w, g->d_speed, g->d_xi);
    YK_LAUNCH(k_particle_info, g->np, 256, 0, st, g->np, g->npp, d_parts, g->d_w, g->d_part,
              g->d_c32, g->d_r32);
    for (auto& L : g->lists) L.valid = false;   // particle pairs change when particles move
    g->nbr_valid = false;
    for (auto& B : g->bands) B.valid = false;
    YK_TRY_CUDA(cudaGetLastError());
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    dev_free(d_parts, st);
    return YK_OK;
}

int build_geometry(yk_geom* g) {
    cudaStream_t st = g->ctx->stream;
    const yk_params& P = g->prm;
    const int os = P.oversample;
    YK_LAUNCH(k_gauss_legendre, 1, 32, 0, st, g->ngl, g->d_glx, g->d_glw);
    YK_LAUNCH(k_ref_matrices, 1, 256, 0, st, g->ngl, os, g->d_glx, g->d_glw, g->d_fine_x,
              g->d_fine_w, g->d_interp, g->d_diff);
    YK_TRY(update_nodes(g));
    const int nf = g->n_near * os * g->ngl;
    const size_t smem = 2 * sizeof(double) * nf;
    if (smem > 48 * 1024)
        YK_TRY_CUDA(cudaFuncSetAttribute(k_qbx_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    dim3 grid(g->npp, g->nshape);
    YK_LAUNCH(k_qbx_rows, grid, 128, smem, st, g->npan, g->ngl, P.near_width, g->n_near, os,
              P.qbx_order, P.qbx_r_factor, P.rho, g->d_shape_ab, g->d_glx, g->d_glw,
              g->d_fine_x, g->d_fine_w, g->d_interp, g->d_cval, g->d_cgrad);
    YK_TRY_CUDA(cudaGetLastError());
    YK_TRY(build_preconditioner(g));
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
