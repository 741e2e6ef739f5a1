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

// P2M: one warp per particle.
// wpp warps per particle, each over every wpp-th group of 32 of its nodes,
// adding its part of the moments to M (zeroed before the launch).
__global__ void k_p2m(GeomView G, const double* __restrict__ sigma, int wpp,
                      double2* __restrict__ M) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= G.np * wpp) return;
    const int p = gw / wpp, part = gw % wpp;
    const d4 c = G.part[p];
    const double rinv = 1.0 / G.rho;
    double mre[EXP_N], mim[EXP_N], I[EXP_N + 1];
    for (int n = 0; n < EXP_N; ++n) mre[n] = mim[n] = 0.0;
    for (int l = 32 * part + lane; l < G.npp; l += 32 * wpp) {
        const int64_t j = (int64_t)p * G.npp + l;
        const double ex = G.x[j] - c.x, ey = G.y[j] - c.y;
        const double s = sqrt(ex * ex + ey * ey);
        const double sinv = 1.0 / s;
        const double esx = ex * sinv, esy = ey * sinv;
        const double a_s = G.nx[j] * esx + G.ny[j] * esy;       // nu . e_s
        const double a_p = -G.nx[j] * esy + G.ny[j] * esx;      // nu . e_phi
        const double ws = G.w[j] * sigma[j];
        bessel_i_down(EXP_ORDER + 1, s * rinv, I);
        double cn = 1.0, sn = 0.0;                               // e^{i n phi}
        for (int n = 0; n <= EXP_ORDER; ++n) {
            const double ip = (n == 0) ? I[1] : 0.5 * (I[n - 1] + I[n + 1]);
            const double ar = a_s * ip * rinv;                   // real part of the bracket
            const double ai = -n * a_p * I[n] * sinv;            // imaginary part
            // e^{-i n phi} (ar + i ai) = (cn - i sn)(ar + i ai)
            mre[n] += ws * (cn * ar + sn * ai);
            mim[n] += ws * (cn * ai - sn * ar);
            const double c2 = cn * esx - sn * esy;
            sn = sn * esx + cn * esy;
            cn = c2;
        }
    }
    for (int n = 0; n <= EXP_ORDER; ++n) {
        double a = mre[n], b = mim[n];
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            double* m = reinterpret_cast<double*>(M + (int64_t)p * EXP_N + n);
            atomicAdd(m, a);
            atomicAdd(m + 1, b);
        }
    }
}

// M2L from the band neighbours of each target particle Q into its local
// coefficients L[Q][m], m = 0..EXP_ORDER (written; zero without neighbours).
// With D = c_Q - c_P = |D| e^{i psi}, Graf's theorem gives
//   L_m = (-1)^m e^{i m psi} sum_{n=-p}^{p} M'_n K_{|n+m|}(|D|/rho),
//   M'_n = M_n e^{i n psi}, M'_{-n} = conj(M'_n):
// the multipole is turned once per pair so that the sum has real weights.
// One block of eight warps per target particle: warp w takes neighbours
// w, w + 8, ... of the list, lane t handles m = t and m = t + 32, and the
// partial expansions are summed in a fixed order at the end.
constexpr int M2L_WARPS = 8;
__global__ void __launch_bounds__(32 * M2L_WARPS) k_band_m2l(GeomView G,
                                                             const double2* __restrict__ M,
                                                             const int* __restrict__ off,
                                                             const int* __restrict__ nbr,
                                                             double2* __restrict__ Lout) {
    __shared__ double Ksh[M2L_WARPS][2 * EXP_ORDER + 1];    // K_k(|D|/rho), k = 0..2p
    __shared__ double2 Msh[M2L_WARPS][EXP_N];               // M'_n, n = 0..p
    __shared__ double2 Lsh[M2L_WARPS][EXP_N];
    const int q = blockIdx.x;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (q >= G.np) return;                                // block-uniform
    double* Kr = Ksh[wib];
    double2* Ms = Msh[wib];
    const int k0 = off[q], k1 = off[q + 1];
    const double rho = G.rho;
    const d4 cq = G.part[q];
    double lr0 = 0.0, li0 = 0.0, lr1 = 0.0, li1 = 0.0;   // m = lane, lane + 32
    for (int k = k0 + wib; k < k1; k += M2L_WARPS) {
        const int p = nbr[k];
        const d4 cp = G.part[p];
        const double Dx = cq.x - cp.x, Dy = cq.y - cp.y;
        const double z = sqrt(Dx * Dx + Dy * Dy) / rho;
        const double psi = atan2(Dy, Dx);
        __syncwarp();
        if (lane == 0) {
            double a, b;
            k01(z, a, b);
            Kr[0] = a;
            Kr[1] = b;
            const double zi2 = 2.0 / z;
            for (int n = 1; n < 2 * EXP_ORDER; ++n) Kr[n + 1] = fma(n * zi2, Kr[n], Kr[n - 1]);
        }
        double2 e[2];                                     // e^{i m psi}, m = lane, lane + 32
        for (int h = 0; h < 2; ++h) {
            const int t = lane + 32 * h;
            if (t > EXP_ORDER) break;
            double s_, c_;
            sincos(t * psi, &s_, &c_);
            e[h] = make_double2(c_, s_);
            const double2 m = M[(int64_t)p * EXP_N + t];
            Ms[t] = make_double2(m.x * c_ - m.y * s_, m.x * s_ + m.y * c_);
        }
        __syncwarp();
        for (int h = 0; h < 2; ++h) {
            const int m = lane + 32 * h;
            if (m > EXP_ORDER) break;
            double lr = Ms[0].x * Kr[m], li = Ms[0].y * Kr[m];
            for (int n = 1; n <= EXP_ORDER; ++n) {
                const double2 Mn = Ms[n];
                const double kp = Kr[n + m], km = Kr[n > m ? n - m : m - n];
                // M'_n K_{n+m} + conj(M'_n) K_{|m-n|}
                lr = fma(Mn.x, kp + km, lr);
                li = fma(Mn.y, kp - km, li);
            }
            const double sg = (m & 1) ? -1.0 : 1.0;
            const double ur = sg * (lr * e[h].x - li * e[h].y);
            const double ui = sg * (lr * e[h].y + li * e[h].x);
            if (h == 0) lr0 += ur, li0 += ui;
            else lr1 += ur, li1 += ui;
        }
    }
    Lsh[wib][lane] = make_double2(lr0, li0);
    if (lane + 32 < EXP_N) Lsh[wib][lane + 32] = make_double2(lr1, li1);
    __syncthreads();
    for (int t = threadIdx.x; t < EXP_N; t += blockDim.x) {
        double2 a = Lsh[0][t];
#pragma unroll
        for (int w = 1; w < M2L_WARPS; ++w) {
            a.x += Lsh[w][t].x;
            a.y += Lsh[w][t].y;
        }
        Lout[(int64_t)q * EXP_N + t] = a;
    }
}

// L2P: value or normal derivative of each node's particle local expansion,
// added to out[] (particles without band neighbours are skipped).
template <bool GRAD>
__global__ void __launch_bounds__(128) k_band_l2p(GeomView G, const double2* __restrict__ Lin,
                                                  const int* __restrict__ off,
                                                  double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= G.n) return;
    const int q = (int)(i / G.npp);
    if (off[q] == off[q + 1]) return;
    const double2* L = Lin + (int64_t)q * EXP_N;
    const d4 cq = G.part[q];
    const double rinv = 1.0 / G.rho;
    const double vx = G.x[i] - cq.x, vy = G.y[i] - cq.y;
    const double r = sqrt(vx * vx + vy * vy);
    const double r_inv = 1.0 / r;
    const double erx = vx * r_inv, ery = vy * r_inv;
    double I[EXP_N + 1];
    bessel_i_down(EXP_ORDER + 1, r * rinv, I);
    double nr = 0.0, nt = 0.0;
    if (GRAD) {
        nr = G.nx[i] * erx + G.ny[i] * ery;        // nu . e_r
        nt = -G.nx[i] * ery + G.ny[i] * erx;       // nu . e_theta
    }
    double acc = 0.0;
    double cm = 1.0, sm = 0.0;                     // (cos, sin)(m theta)
    for (int m = 0; m <= EXP_ORDER; ++m) {
        const double2 Lm = L[m];
        // z = L_m e^{-i m theta}; Re[z X] with X real (value) or complex (gradient)
        const double zr = Lm.x * cm + Lm.y * sm, zi = Lm.y * cm - Lm.x * sm;
        double term;
        if (!GRAD) {
            term = zr * I[m];
        } else {
            const double ip = (m == 0) ? I[1] : 0.5 * (I[m - 1] + I[m + 1]);
            const double xr = nr * ip * rinv;      // X = nu.e_r I_m'/rho - i m nu.e_theta I_m/r
            const double xi = -m * nt * I[m] * r_inv;
            term = zr * xr - zi * xi;
        }
        acc += (m == 0 ? 1.0 : 2.0) * term;
        const double c2 = cm * erx - sm * ery;
        sm = sm * erx + cm * ery;
        cm = c2;
    }
    out[i] += acc / (2.0 * PI);
}

// Band lists per target particle: source particles P != Q with
// lo <= gap(P, Q) < hi (bounding circles), as CSR.
__device__ __forceinline__ bool gap_below(const d4& a, const d4& b, double thr) {
    const double dx = __dsub_rn(a.x, b.x), dy = __dsub_rn(a.y, b.y);
    const double s = __dadd_rn(__dadd_rn(a.z, b.z), thr);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) < __dmul_rn(s, s);
}

// One warp per target particle Q, lanes over P; the fill writes in order of P.
__global__ void k_band_count(int np, const d4* __restrict__ part, double lo, double hi, int* counts) {
    const int Q = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (Q >= np) return;   // warp-uniform
    const d4 a = part[Q];
    int c = 0;
    for (int P0 = 0; P0 < np; P0 += 32) {
        const int P = P0 + lane;
        const bool hit = P < np && P != Q && !gap_below(a, part[P], lo) && gap_below(a, part[P], hi);
        c += __popc(__ballot_sync(0xffffffffu, hit));
    }
    if (lane == 0) counts[Q] = c;
}

__global__ void k_band_fill(int np, const d4* __restrict__ part, double lo, double hi,
                            const int* __restrict__ off, int* __restrict__ nbr) {
    const int Q = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (Q >= np) return;   // warp-uniform
    const d4 a = part[Q];
    int k = off[Q];
    for (int P0 = 0; P0 < np; P0 += 32) {
        const int P = P0 + lane;
        const bool hit = P < np && P != Q && !gap_below(a, part[P], lo) && gap_below(a, part[P], hi);
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) nbr[k + __popc(m & ((1u << lane) - 1u))] = P;
        k += __popc(m);
    }
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
    YK_LAUNCH(k_band_count, ceil_div(g->np, 4), 128, 0, st, g->np, g->d_part, lo, hi, counts);
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
        YK_LAUNCH(k_band_fill, ceil_div(g->np, 4), 128, 0, st, g->np, g->d_part, lo, hi, B.off,
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
    // warps per particle: enough for about 32 warps per SM in all
    const int wpp = std::max(1, std::min(ceil_div(152 * 32, g->np), ceil_div(g->npp, 32)));
    YK_TRY_CUDA(cudaMemsetAsync(g->d_mpole, 0, sizeof(double2) * (size_t)g->np * EXP_N, st));
    YK_LAUNCH(k_p2m, ceil_div((int64_t)g->np * wpp * 32, 128), 128, 0, st, G, sigma, wpp,
              g->d_mpole);
    YK_LAUNCH(k_band_m2l, g->np, 32 * M2L_WARPS, 0, st, G, g->d_mpole, g->bands[kind].off,
              g->bands[kind].idx, g->d_local);
    if (grad)
        YK_LAUNCH(k_band_l2p<true>, ceil_div(g->n, 128), 128, 0, st, G, g->d_local,
                  g->bands[kind].off, out);
    else
        YK_LAUNCH(k_band_l2p<false>, ceil_div(g->n, 128), 128, 0, st, G, g->d_local,
                  g->bands[kind].off, out);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

}  // namespace yk
