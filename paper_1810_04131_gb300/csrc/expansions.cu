// FP64 particle expansions for the middle band of the precision-split
// operators: source particles whose gap to the target particle lies in
// [expansion gap, split gap) (too close for FP32, far enough for a
// converging expansion).
//
// Graf's addition theorem (Section 5, Eq. graf-addition, Yukawa form via
// K0(z) = (i pi/2) H0(iz)) gives, for |y - c| < |x - c|,
//   K0(|x - y|/rho) = sum_n K_n(|x - c|/rho) I_n(|y - c|/rho) e^{i n (theta_x - phi_y)},
// so the double-layer potential of particle P (centre c_P) at x outside it is
//   u_P(x) = (1/2pi) sum_n M_n K_n(|x - c_P|/rho) e^{i n theta_x},
//   M_n = sum_j w_j sigma_j e^{-i n phi_j} [(nu.e_s) I_n'(s_j/rho)/rho - i n (nu.e_phi) I_n(s_j/rho)/s_j]
// (P2M; M_{-n} = conj M_n). With D = c_Q - c_P and v = x - c_Q, |v| < |D|,
//   K_n(|D + v|/rho) e^{i n arg(D+v)} = sum_m (-1)^m K_{n+m}(|D|/rho) I_m(|v|/rho)
//                                       e^{i (n+m) arg D} e^{-i m arg v},
// so u_P(x) = (1/2pi) sum_m L_m I_m(|v|/rho) e^{-i m arg v} with
//   L_m = sum_n M_n (-1)^m K_{n+m}(|D|/rho) e^{i (n+m) arg D}   (M2L; L_{-m} = conj L_m)
// and the target values follow (L2P), or their normal derivative with
// grad[I_m(r/rho) e^{-i m theta}] = e^{-i m theta}[I_m'/rho e_r - i m I_m/r e_theta].
// With bounding radii R and gap g the terms decay like (2R/(2R + g))^{n+m}.
#include <math.h>

#include <algorithm>

#include "bessel.cuh"
#include "yk_internal.cuh"

namespace yk {

constexpr int EXP_ORDER = EXPANSION_TERMS - 1;   // terms |n|, |m| <= EXP_ORDER
constexpr int EXP_N = EXPANSION_TERMS;

// I_0..I_{EXP_ORDER+1}(x) for 0 < x (series for the top two orders, then the
// backward recurrence I_{k-1} = I_{k+1} + (2k/x) I_k, stable downwards).
__device__ inline void bessel_i_all(double x, double* I) {
    const int top = EXP_ORDER + 1;
    I[top] = bessel_i_series(top, x);
    I[top - 1] = bessel_i_series(top - 1, x);
    for (int k = top - 1; k >= 1; --k) I[k - 1] = I[k + 1] + (2.0 * k / x) * I[k];
}

// P2M: one warp per particle.
__global__ void k_p2m(GeomView G, const double* __restrict__ sigma, double2* __restrict__ M) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= G.np) return;
    const int p = warp;
    const d4 c = G.part[p];
    const double rho = G.rho;
    double mre[EXP_N], mim[EXP_N], I[EXP_N + 1];
    for (int n = 0; n < EXP_N; ++n) mre[n] = mim[n] = 0.0;
    for (int l = lane; l < G.npp; l += 32) {
        const int64_t j = (int64_t)p * G.npp + l;
        const double ex = G.x[j] - c.x, ey = G.y[j] - c.y;
        const double s = sqrt(ex * ex + ey * ey);
        const double esx = ex / s, esy = ey / s;
        const double a_s = G.nx[j] * esx + G.ny[j] * esy;       // nu . e_s
        const double a_p = -G.nx[j] * esy + G.ny[j] * esx;      // nu . e_phi
        const double ws = G.w[j] * sigma[j];
        bessel_i_all(s / rho, I);
        double cph = esx, sph = esy;                             // e^{i phi}
        double cn = 1.0, sn = 0.0;                               // e^{i n phi}
        for (int n = 0; n <= EXP_ORDER; ++n) {
            const double ip = (n == 0) ? I[1] : 0.5 * (I[n - 1] + I[n + 1]);
            const double ar = a_s * ip / rho;                    // real part of the bracket
            const double ai = -n * a_p * I[n] / s;               // imaginary part
            // e^{-i n phi} (ar + i ai) = (cn - i sn)(ar + i ai)
            mre[n] += ws * (cn * ar + sn * ai);
            mim[n] += ws * (cn * ai - sn * ar);
            const double c2 = cn * cph - sn * sph;
            sn = sn * cph + cn * sph;
            cn = c2;
        }
    }
    for (int n = 0; n <= EXP_ORDER; ++n) {
        double a = mre[n], b = mim[n];
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) M[(int64_t)p * EXP_N + n] = make_double2(a, b);
    }
}

// M2L from the band neighbours of target particle Q, then L2P (value or
// normal derivative), added to out[]. One CTA per target particle.
template <bool GRAD>
__global__ void __launch_bounds__(256) k_m2l_l2p(GeomView G, const double2* __restrict__ M,
                                                 const int* __restrict__ off,
                                                 const int* __restrict__ nbr,
                                                 double* __restrict__ out) {
    const int q = blockIdx.x;
    const int k0 = off[q], k1 = off[q + 1];
    if (k0 == k1) return;                       // uniform: no band neighbours
    __shared__ double Kr[2 * EXP_ORDER + 1];    // K_k(|D|/rho), k = 0..2p
    __shared__ double2 eps[3 * EXP_ORDER + 1];  // e^{i k psi}, k = -p..2p
    __shared__ double2 Ms[EXP_N];
    __shared__ double2 L[EXP_N];
    const double rho = G.rho;
    const d4 cq = G.part[q];
    if (threadIdx.x < EXP_N) L[threadIdx.x] = make_double2(0.0, 0.0);
    for (int k = k0; k < k1; ++k) {
        const int p = nbr[k];
        const d4 cp = G.part[p];
        const double Dx = cq.x - cp.x, Dy = cq.y - cp.y;
        const double Dn = sqrt(Dx * Dx + Dy * Dy);
        const double psi = atan2(Dy, Dx);
        __syncthreads();
        if (threadIdx.x == 0) {
            const double z = Dn / rho;
            double a, b;
            k01(z, a, b);
            Kr[0] = a;
            Kr[1] = b;
            for (int n = 1; n < 2 * EXP_ORDER; ++n) Kr[n + 1] = Kr[n - 1] + (2.0 * n / z) * Kr[n];
        }
        for (int t = threadIdx.x; t < 3 * EXP_ORDER + 1; t += blockDim.x) {
            double s_, c_;
            sincos((t - EXP_ORDER) * psi, &s_, &c_);
            eps[t] = make_double2(c_, s_);
        }
        if (threadIdx.x < EXP_N) Ms[threadIdx.x] = M[(int64_t)p * EXP_N + threadIdx.x];
        __syncthreads();
        if (threadIdx.x < EXP_N) {
            const int m = threadIdx.x;
            double lr = 0.0, li = 0.0;
            for (int n = -EXP_ORDER; n <= EXP_ORDER; ++n) {
                const double2 Mn = n >= 0 ? Ms[n] : make_double2(Ms[-n].x, -Ms[-n].y);
                const int kk = n + m;                            // in [-p, 2p]
                const double Kv = Kr[kk < 0 ? -kk : kk];
                const double2 e = eps[kk + EXP_ORDER];
                // M_n * K * e^{i (n+m) psi}
                lr += Kv * (Mn.x * e.x - Mn.y * e.y);
                li += Kv * (Mn.x * e.y + Mn.y * e.x);
            }
            const double sg = (m & 1) ? -1.0 : 1.0;
            L[m].x += sg * lr;
            L[m].y += sg * li;
        }
    }
    __syncthreads();
    // L2P
    double I[EXP_N + 1];
    for (int l = threadIdx.x; l < G.npp; l += blockDim.x) {
        const int64_t i = (int64_t)q * G.npp + l;
        const double vx = G.x[i] - cq.x, vy = G.y[i] - cq.y;
        const double r = sqrt(vx * vx + vy * vy);
        const double erx = vx / r, ery = vy / r;
        bessel_i_all(r / rho, I);
        double nr = 0.0, nt = 0.0;
        if (GRAD) {
            nr = G.nx[i] * erx + G.ny[i] * ery;        // nu . e_r
            nt = -G.nx[i] * ery + G.ny[i] * erx;       // nu . e_theta
        }
        double acc = 0.0;
        double cm = 1.0, sm = 0.0;                     // e^{-i m theta} = cm - i sm... (cos, sin of m theta)
        for (int m = 0; m <= EXP_ORDER; ++m) {
            const double2 Lm = L[m];
            // Re[L_m e^{-i m theta} X] with X real (value) or complex (gradient)
            const double er = cm, ei = -sm;            // e^{-i m theta}
            const double zr = Lm.x * er - Lm.y * ei, zi = Lm.x * ei + Lm.y * er;
            double term;
            if (!GRAD) {
                term = zr * I[m];
            } else {
                const double ip = (m == 0) ? I[1] : 0.5 * (I[m - 1] + I[m + 1]);
                const double xr = nr * ip / rho;       // X = nu.e_r I_m'/rho - i m nu.e_theta I_m/r
                const double xi = -m * nt * I[m] / r;
                term = zr * xr - zi * xi;
            }
            acc += (m == 0 ? 1.0 : 2.0) * term;
            const double c2 = cm * erx - sm * ery;     // advance (cos, sin)(m theta)
            sm = sm * erx + cm * ery;
            cm = c2;
        }
        out[i] += acc / (2.0 * PI);
    }
}

// Band lists per target particle: source particles P != Q with
// lo <= gap(P, Q) < hi (bounding circles), as CSR.
__device__ __forceinline__ bool gap_below(const d4& a, const d4& b, double thr) {
    const double dx = __dsub_rn(a.x, b.x), dy = __dsub_rn(a.y, b.y);
    const double s = __dadd_rn(__dadd_rn(a.z, b.z), thr);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) < __dmul_rn(s, s);
}

__global__ void k_band_count(int np, const d4* __restrict__ part, double lo, double hi, int* counts) {
    const int Q = blockIdx.x * blockDim.x + threadIdx.x;
    if (Q >= np) return;
    const d4 a = part[Q];
    int c = 0;
    for (int P = 0; P < np; ++P)
        c += (P != Q && !gap_below(a, part[P], lo) && gap_below(a, part[P], hi)) ? 1 : 0;
    counts[Q] = c;
}

__global__ void k_band_fill(int np, const d4* __restrict__ part, double lo, double hi,
                            const int* __restrict__ off, int* __restrict__ nbr) {
    const int Q = blockIdx.x * blockDim.x + threadIdx.x;
    if (Q >= np) return;
    const d4 a = part[Q];
    int k = off[Q];
    for (int P = 0; P < np; ++P)
        if (P != Q && !gap_below(a, part[P], lo) && gap_below(a, part[P], hi)) nbr[k++] = P;
}

__global__ void k_scan_counts(int np, const int* __restrict__ counts, int* __restrict__ off) {
    __shared__ int buf[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b = 0; b < np; b += 1024) {
        const int i = b + threadIdx.x;
        buf[threadIdx.x] = (i < np) ? counts[i] : 0;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int v = (threadIdx.x >= o) ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += v;
            __syncthreads();
        }
        if (i < np) off[i + 1] = carry + buf[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 1023) carry += buf[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) off[0] = 0;
}

static int band_list(yk_geom* g, int kind, double lo, double hi) {
    BandList& B = g->bands[kind];
    if (B.valid) return YK_OK;
    cudaStream_t st = g->ctx->stream;
    if (!B.off) YK_TRY(dev_alloc((void**)&B.off, sizeof(int) * (g->np + 1), st));
    int* counts = g->d_counts;
    YK_LAUNCH(k_band_count, ceil_div(g->np, 128), 128, 0, st, g->np, g->d_part, lo, hi, counts);
    YK_LAUNCH(k_scan_counts, 1, 1024, 0, st, g->np, counts, B.off);
    int total = 0;
    YK_TRY_CUDA(cudaMemcpyAsync(&total, B.off + g->np, sizeof(int), cudaMemcpyDeviceToHost, st));
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    if (total > B.cap) {
        dev_free(B.idx, st);
        B.idx = nullptr;
        B.cap = 0;
        YK_TRY(dev_alloc((void**)&B.idx, sizeof(int) * (size_t)std::max(total, 1), st));
        B.cap = std::max(total, 1);
    }
    if (total > 0)
        YK_LAUNCH(k_band_fill, ceil_div(g->np, 128), 128, 0, st, g->np, g->d_part, lo, hi, B.off,
                  B.idx);
    YK_TRY_CUDA(cudaGetLastError());
    B.n = total;
    B.valid = true;
    return YK_OK;
}

// Add the band's contribution (value or normal derivative) to out.
int band_expansions(yk_geom* g, const double* sigma, double* out, bool grad) {
    const int kind = grad ? 1 : 0;
    const double lo = grad ? g->tile_gap_grad : g->tile_gap;
    const double hi = grad ? g->split_gap_grad : g->split_gap;
    if (!(hi > lo)) return YK_OK;
    YK_TRY(band_list(g, kind, lo, hi));
    if (g->bands[kind].n == 0) return YK_OK;
    cudaStream_t st = g->ctx->stream;
    GeomView G = g->view();
    YK_LAUNCH(k_p2m, ceil_div((int64_t)g->np * 32, 128), 128, 0, st, G, sigma, g->d_mpole);
    if (grad)
        YK_LAUNCH(k_m2l_l2p<true>, g->np, 256, 0, st, G, g->d_mpole, g->bands[kind].off,
                  g->bands[kind].idx, out);
    else
        YK_LAUNCH(k_m2l_l2p<false>, g->np, 256, 0, st, G, g->d_mpole, g->bands[kind].off,
                  g->bands[kind].idx, out);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

}  // namespace yk
