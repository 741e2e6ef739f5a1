// Coarse-space deflation of the inner (FP32) GMRES of the mixed solve of
// 1/2 sigma + D sigma = f (Eq. bie).
//
// The block preconditioner M (the inverse own-particle blocks) leaves the
// coupling between particles to GMRES, and what it converges slowest on are
// the lowest Fourier modes of each particle's density, the ones its
// neighbours see as its charge and dipole. The coarse space Z holds three
// modes per particle P: 1, cos(theta), sin(theta) of the polar angle of its
// nodes about its centre, orthonormalised over P's nodes. GMRES runs on the
// deflated operator
//     B P v = B v - (B Z) C Z^T (B v - v),   B = A M,   C = (Z^T B Z)^{-1},
// P = I - Z C Z^T B + Z C Z^T, whose coarse components are exact
// (Z^T B P = Z^T); a cycle's correction is x += M P y with
// P y = y - Z C Z^T (B y - y), and Z^T (B y - y) is the combination of the
// Z^T (B v_j - v_j) kept from the Arnoldi steps, so B P costs one operator
// application, like B. With the kept z_j = M v_j of the GMRES, M P y is
// Z_kept y - (M Z) C sum_j y_j Z^T (B v_j - v_j).
//
// B Z is stored. Its column for mode c of particle Q is A (M Z_Q): on Q's
// own nodes the own-particle part of the FP32 operator (self block and QBX
// rows), on the nodes of another particle P the plain quadrature of the
// double-layer kernel over Q's nodes, in the FP32 arithmetic of the far-field
// kernels. Only source particles Q whose whole contribution at P is bounded
// above COARSE_TOL x max|sigma| are kept (the K1 kernel decays like
// exp(-r/rho)): per target particle P a CSR list of (P, Q) entries, each with
// a [3][npp] block. Z^T B Z (3 np square, 3 x 3 blocks per entry) is
// inverted once per configuration by blocked Gauss-Jordan (panels of 16
// particles); a pivot that is numerically zero turns the deflation off for
// that configuration.
//
// Per Arnoldi step: u_j = Z^T (w - v_j) (one block per particle),
// c = C u_j (one warp per row), w -= (B Z) c (one block per target
// particle over its entries); per cycle x -= (M Z) C sum_j y_j u_j.
#include <math.h>

#include <algorithm>

#include "p2p_kernels.cuh"
#include "yk_internal.cuh"

namespace yk {

constexpr int CO_TPB = 256;

// ---------------------------------------------------------------------------
// Setup kernels

// Source particle Q couples to target particle P (or Q == P).
__device__ __forceinline__ bool coarse_coupled(const d4& a, const d4& b, double gap) {
    const double dx = a.x - b.x, dy = a.y - b.y;
    return sqrt(dx * dx + dy * dy) - a.z - b.z < gap;
}

// One warp per target particle P: counts[P] = coupled Q (P included).
__global__ void k_coarse_count(int np, const d4* __restrict__ part, double gap,
                               int* __restrict__ counts) {
    const int P = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (P >= np) return;   // P is uniform over the warp
    const d4 a = part[P];
    int c = 0;
    for (int Q0 = 0; Q0 < np; Q0 += 32) {
        const int Q = Q0 + lane;
        const bool in = Q < np && (Q == P || coarse_coupled(a, part[Q], gap));
        c += __popc(__ballot_sync(0xffffffffu, in));
    }
    if (lane == 0) counts[P] = c;
}

// off[0] = 0, off[P + 1] = off[P] + counts[P] (np <= COARSE_MAX_PARTICLES).
__global__ void k_coarse_scan(int np, const int* __restrict__ counts, int* __restrict__ off) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int s = 0;
    off[0] = 0;
    for (int P = 0; P < np; ++P) {
        s += counts[P];
        off[P + 1] = s;
    }
}

// The entries (P, Q) of target particle P in increasing Q.
__global__ void k_coarse_fill(int np, const d4* __restrict__ part, double gap,
                              const int* __restrict__ off, int2* __restrict__ ent) {
    const int P = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (P >= np) return;
    const d4 a = part[P];
    int pos = off[P];
    for (int Q0 = 0; Q0 < np; Q0 += 32) {
        const int Q = Q0 + lane;
        const bool in = Q < np && (Q == P || coarse_coupled(a, part[Q], gap));
        const unsigned b = __ballot_sync(0xffffffffu, in);
        if (in) ent[pos + __popc(b & ((1u << lane) - 1u))] = make_int2(P, Q);
        pos += __popc(b);
    }
}

template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* red /* [K][CO_TPB / 32] */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[k * (CO_TPB / 32) + wid] = x;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double x = 0.0;
        for (int w = 0; w < CO_TPB / 32; ++w) x += red[k * (CO_TPB / 32) + w];
        v[k] = x;
    }
    __syncthreads();
}

// One block per particle: Z_c (c = 0, 1, 2) from 1, cos(theta), sin(theta)
// of the polar angle about the centre, orthonormalised over the particle's
// nodes by the Cholesky factor of their Gram matrix.
__global__ void __launch_bounds__(CO_TPB) k_coarse_modes(GeomView G, double* __restrict__ Z) {
    __shared__ double red[5 * (CO_TPB / 32)];
    const int p = blockIdx.x;
    const int64_t base = (int64_t)p * G.npp;
    const d4 c = G.part[p];
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // sum cos, sin, cos^2, cos sin, sin^2
    for (int t = threadIdx.x; t < G.npp; t += CO_TPB) {
        const double dx = G.x[base + t] - c.x, dy = G.y[base + t] - c.y;
        const double ri = 1.0 / sqrt(dx * dx + dy * dy);
        const double co = dx * ri, si = dy * ri;
        s[0] += co;
        s[1] += si;
        s[2] += co * co;
        s[3] += co * si;
        s[4] += si * si;
    }
    block_sum<5>(s, red);
    // Gram matrix of (1, cos, sin) = L L^T
    const double l00 = sqrt((double)G.npp);
    const double l10 = s[0] / l00, l20 = s[1] / l00;
    const double l11 = sqrt(fmax(s[2] - l10 * l10, 0.0));
    const double l21 = (s[3] - l20 * l10) / l11;
    const double l22 = sqrt(fmax(s[4] - l20 * l20 - l21 * l21, 0.0));
    for (int t = threadIdx.x; t < G.npp; t += CO_TPB) {
        const double dx = G.x[base + t] - c.x, dy = G.y[base + t] - c.y;
        const double ri = 1.0 / sqrt(dx * dx + dy * dy);
        const double q0 = 1.0 / l00;
        const double q1 = (dx * ri - l10 * q0) / l11;
        const double q2 = (dy * ri - l20 * q0 - l21 * q1) / l22;
        Z[base + t] = q0;
        Z[G.n + base + t] = q1;
        Z[2 * G.n + base + t] = q2;
    }
}

// One block per entry e = (P, Q): W_e[c][t] = (B Z_{Q,c}) at node t of P,
// and the 3 x 3 block Z_P^T W_e of Z^T B Z (row-major, nc columns).
// Y = M Z ([3][n]); O = the own-particle part of A Y ([3][n]). The far
// pairs use the FP32 far-field kernel's arithmetic: coordinates relative to
// the source centre scaled by kpf = log2(e)/rho, radial factor coef_any,
// and ks = sqrt(log2 e)/(2 pi rho) (see PairF32).
__global__ void __launch_bounds__(CO_TPB)
    k_coarse_blocks(GeomView G, const int2* __restrict__ ent, const double* __restrict__ Y,
                    const double* __restrict__ O, const double* __restrict__ Z, float kpf, float ks,
                    float* __restrict__ W, float* __restrict__ Cm, int nc) {
    extern __shared__ float4 srec[];   // [2 npp]: (xs, ys, gx0, gy0), (gx1, gy1, gx2, gy2)
    __shared__ double red[9 * (CO_TPB / 32)];
    const int e = blockIdx.x;
    const int2 pq = ent[e];
    const int P = pq.x, Q = pq.y;
    const int npp = G.npp;
    const int64_t n = G.n;
    const int64_t bp = (int64_t)P * npp, bq = (int64_t)Q * npp;
    float* We = W + (int64_t)e * 3 * npp;
    double acc[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // [a][c]
    if (P == Q) {
        for (int t = threadIdx.x; t < npp; t += CO_TPB) {
            float wv[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                wv[c] = (float)O[c * n + bp + t];
                We[c * npp + t] = wv[c];
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double za = Z[a * n + bp + t];
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[3 * a + c] += za * (double)wv[c];
            }
        }
    } else {
        for (int s = threadIdx.x; s < npp; s += CO_TPB) {
            const int64_t j = bq + s;
            const float2 xq = G.xi[j];
            const double wn = G.w[j];
            float g[6];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double ws = wn * Y[c * n + j];
                g[2 * c] = (float)(ws * G.nx[j]);
                g[2 * c + 1] = (float)(ws * G.ny[j]);
            }
            srec[2 * s] = make_float4(-kpf * xq.x, -kpf * xq.y, g[0], g[1]);
            srec[2 * s + 1] = make_float4(g[2], g[3], g[4], g[5]);
        }
        __syncthreads();
        const float4 ct = G.c32[P], cs = G.c32[Q];
        const float dXc = kpf * ((ct.x - cs.x) + (ct.z - cs.z));
        const float dYc = kpf * ((ct.y - cs.y) + (ct.w - cs.w));
        for (int t = threadIdx.x; t < npp; t += CO_TPB) {
            const float2 xt = G.xi[bp + t];
            const float TX = fmaf(kpf, xt.x, dXc), TY = fmaf(kpf, xt.y, dYc);
            float f0 = 0.0f, f1 = 0.0f, f2 = 0.0f;
            for (int s = 0; s < npp; ++s) {
                const float4 A = srec[2 * s], B = srec[2 * s + 1];
                const float dX = TX + A.x, dY = TY + A.y;
                const float k = coef_any(dX, dY);
                f0 = fmaf(k, fmaf(dX, A.z, dY * A.w), f0);
                f1 = fmaf(k, fmaf(dX, B.x, dY * B.y), f1);
                f2 = fmaf(k, fmaf(dX, B.z, dY * B.w), f2);
            }
            const float wv[3] = {f0 * ks, f1 * ks, f2 * ks};
#pragma unroll
            for (int c = 0; c < 3; ++c) We[c * npp + t] = wv[c];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double za = Z[a * n + bp + t];
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[3 * a + c] += za * (double)wv[c];
            }
        }
    }
    block_sum<9>(acc, red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Cm[(int64_t)(3 * P + a) * nc + 3 * Q + c] = (float)acc[3 * a + c];
    }
}

// Blocked in-place Gauss-Jordan inversion of M (nc x nc, row-major), panel
// by panel: with the pivot block K = [k0, k0 + w) and D = M_KK,
//   M_KK <- D^{-1},  M_Kj <- D^{-1} M_Kj,  M_iK <- -M_iK D^{-1},
//   M_ij <- M_ij - M_iK D^{-1} M_Kj   (i, j outside K),
// which after the last panel leaves M^{-1}. Per panel: D^{-1} by scalar
// Gauss-Jordan in one block (k_gj_pivot), the copies Cp = M_:K and
// R = D^{-1} M_K: (k_gj_panel), then the update of every entry
// (k_gj_update). No pivoting: Z^T B Z is the identity plus the couplings
// between particles' modes; a pivot not above 1e-6 x its row's largest
// entry sets *flag.
constexpr int GJ_W = 48;       // panel width (16 particles)
constexpr int GJ_ROWS = 32;    // rows per block of the update
constexpr int GJ_COLS = 128;   // columns (threads) per block of the update
constexpr int GJ_PTPB = 64;    // threads per block of the panel copies
constexpr int GJ_PROWS = 8;    // rows of R per block of the panel copies

// D^{-1} of the panel's diagonal block by in-place Gauss-Jordan over its
// 3 x 3 pivot blocks (the formulas above with w = 3), in shared memory.
// A pivot block whose determinant is not above 1e-6 x the product of its
// row norms sets *flag.
__global__ void __launch_bounds__(CO_TPB)
    k_gj_pivot(int nc, int k0, int w, const float* __restrict__ M, float* __restrict__ Dinv,
               int* __restrict__ flag) {
    constexpr int PER = (GJ_W * GJ_W + CO_TPB - 1) / CO_TPB;
    __shared__ float D[GJ_W * GJ_W];
    __shared__ float prow[3 * GJ_W], pcol[3 * GJ_W];
    int ra[PER], ca[PER];   // this thread's entries
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int t = threadIdx.x + u * CO_TPB;
        ra[u] = t < w * w ? t / w : -1;
        ca[u] = t < w * w ? t % w : 0;
        if (ra[u] >= 0) D[t] = M[(int64_t)(k0 + ra[u]) * nc + k0 + ca[u]];
    }
    __syncthreads();
    for (int s0 = 0; s0 < w; s0 += 3) {
        for (int t = threadIdx.x; t < 3 * w; t += CO_TPB) {
            const int a = t / w, c = t % w;
            prow[t] = D[(s0 + a) * w + c];        // [a][c]
            pcol[t] = D[c * w + s0 + a];          // [a][c] = D[c][s0 + a]
        }
        __syncthreads();
        // every thread forms Q = adj / det of the pivot block itself
        float q[9];
        {
            float p[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) p[a][b] = prow[a * w + s0 + b];
            const float c00 = p[1][1] * p[2][2] - p[1][2] * p[2][1];
            const float c01 = p[1][2] * p[2][0] - p[1][0] * p[2][2];
            const float c02 = p[1][0] * p[2][1] - p[1][1] * p[2][0];
            const float det = p[0][0] * c00 + p[0][1] * c01 + p[0][2] * c02;
            float rn2 = 1.0f;
#pragma unroll
            for (int a = 0; a < 3; ++a) rn2 *= p[a][0] * p[a][0] + p[a][1] * p[a][1] + p[a][2] * p[a][2];
            const bool bad = !(det * det > 1e-12f * rn2);
            if (bad && threadIdx.x == 0) *flag = 1;
            const float di = bad ? 0.0f : 1.0f / det;
            q[0] = c00 * di;
            q[3] = c01 * di;
            q[6] = c02 * di;
            q[1] = (p[0][2] * p[2][1] - p[0][1] * p[2][2]) * di;
            q[4] = (p[0][0] * p[2][2] - p[0][2] * p[2][0]) * di;
            q[7] = (p[0][1] * p[2][0] - p[0][0] * p[2][1]) * di;
            q[2] = (p[0][1] * p[1][2] - p[0][2] * p[1][1]) * di;
            q[5] = (p[0][2] * p[1][0] - p[0][0] * p[1][2]) * di;
            q[8] = (p[0][0] * p[1][1] - p[0][1] * p[1][0]) * di;
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int a = ra[u], c = ca[u];
            if (a < 0) continue;
            const int ib = a - s0, jb = c - s0;
            const bool ri = (unsigned)ib < 3u, cj = (unsigned)jb < 3u;
            float t0, t1, t2;   // row ib of Q, or D_aK Q
            if (ri) {
                t0 = ib == 0 ? q[0] : (ib == 1 ? q[3] : q[6]);
                t1 = ib == 0 ? q[1] : (ib == 1 ? q[4] : q[7]);
                t2 = ib == 0 ? q[2] : (ib == 1 ? q[5] : q[8]);
            } else {
                const float m0 = pcol[a], m1 = pcol[w + a], m2 = pcol[2 * w + a];
                t0 = m0 * q[0] + m1 * q[3] + m2 * q[6];
                t1 = m0 * q[1] + m1 * q[4] + m2 * q[7];
                t2 = m0 * q[2] + m1 * q[5] + m2 * q[8];
            }
            float v;
            if (cj) {
                const float tj = jb == 0 ? t0 : (jb == 1 ? t1 : t2);
                v = ri ? tj : -tj;
            } else {
                const float sum = t0 * prow[c] + t1 * prow[w + c] + t2 * prow[2 * w + c];
                v = ri ? sum : D[a * w + c] - sum;
            }
            D[a * w + c] = v;
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < PER; ++u)
        if (ra[u] >= 0) Dinv[ra[u] * w + ca[u]] = D[ra[u] * w + ca[u]];
}

// Blocks of GJ_PTPB columns q x GJ_PROWS rows b:
// R[b][q] = sum_c Dinv[b][c] M[k0 + c][q] and Cp[q][b] = M[q][k0 + b],
// both from the pre-step M.
__global__ void __launch_bounds__(GJ_PTPB)
    k_gj_panel(int nc, int k0, int w, const float* __restrict__ M, const float* __restrict__ Dinv,
               float* __restrict__ Cp, float* __restrict__ R) {
    __shared__ float Ds[GJ_PROWS * GJ_W];
    const int b0 = blockIdx.y * GJ_PROWS;
    for (int t = threadIdx.x; t < GJ_PROWS * GJ_W; t += GJ_PTPB) {
        const int b = b0 + t / GJ_W, c = t % GJ_W;
        Ds[t] = (b < w && c < w) ? Dinv[b * w + c] : 0.0f;
    }
    __syncthreads();
    const int q = blockIdx.x * GJ_PTPB + threadIdx.x;
    if (q >= nc) return;
    float m[GJ_W];
#pragma unroll
    for (int c = 0; c < GJ_W; ++c) m[c] = c < w ? M[(int64_t)(k0 + c) * nc + q] : 0.0f;
#pragma unroll
    for (int r = 0; r < GJ_PROWS; ++r) {
        const int b = b0 + r;
        if (b >= w) break;
        float acc = 0.0f;
#pragma unroll
        for (int c = 0; c < GJ_W; ++c) acc = fmaf(Ds[r * GJ_W + c], m[c], acc);
        R[(int64_t)b * nc + q] = acc;
        Cp[(int64_t)q * GJ_W + b] = M[(int64_t)q * nc + k0 + b];
    }
}

// GJ_ROWS rows x GJ_COLS columns per block: the panel's update of M.
__global__ void __launch_bounds__(GJ_COLS)
    k_gj_update(int nc, int k0, int w, float* __restrict__ M, const float* __restrict__ Dinv,
                const float* __restrict__ Cp, const float* __restrict__ R) {
    __shared__ float cps[GJ_ROWS * GJ_W];
    const int i0 = blockIdx.y * GJ_ROWS;
    for (int t = threadIdx.x; t < GJ_ROWS * GJ_W; t += GJ_COLS) {
        const int a = t / GJ_W, b = t % GJ_W;
        cps[t] = (i0 + a < nc && b < w) ? Cp[(int64_t)(i0 + a) * GJ_W + b] : 0.0f;
    }
    __syncthreads();
    const int j = blockIdx.x * GJ_COLS + threadIdx.x;
    if (j >= nc) return;
    const int jk = j - k0;
    const bool jK = (unsigned)jk < (unsigned)w;
    // column j of D^{-1} (pivot columns) or of R
    float col[GJ_W];
#pragma unroll
    for (int b = 0; b < GJ_W; ++b)
        col[b] = b < w ? (jK ? Dinv[b * w + jk] : R[(int64_t)b * nc + j]) : 0.0f;
    for (int a = 0; a < GJ_ROWS; ++a) {
        const int i = i0 + a;
        if (i >= nc) break;
        float* mij = M + (int64_t)i * nc + j;
        const int ik = i - k0;
        if ((unsigned)ik < (unsigned)w) {   // pivot rows: D^{-1} or R
            *mij = jK ? Dinv[ik * w + jk] : R[(int64_t)ik * nc + j];
        } else {
            float s = 0.0f;
#pragma unroll
            for (int b = 0; b < GJ_W; ++b) s = fmaf(cps[a * GJ_W + b], col[b], s);
            *mij = (jK ? 0.0f : *mij) - s;
        }
    }
}

// ---------------------------------------------------------------------------
// Per-step kernels

// One block per particle: u[3 p + a] = Z_a^T (w - v) over p's nodes.
__global__ void __launch_bounds__(CO_TPB)
    k_coarse_restrict(int npp, int64_t n, const double* __restrict__ Z, const double* __restrict__ w,
                      const double* __restrict__ v, double* __restrict__ u) {
    __shared__ double red[3 * (CO_TPB / 32)];
    const int p = blockIdx.x;
    const int64_t base = (int64_t)p * npp;
    double s[3] = {0.0, 0.0, 0.0};
    for (int t = threadIdx.x; t < npp; t += CO_TPB) {
        const int64_t i = base + t;
        const double d = w[i] - v[i];
        s[0] = fma(Z[i], d, s[0]);
        s[1] = fma(Z[n + i], d, s[1]);
        s[2] = fma(Z[2 * n + i], d, s[2]);
    }
    block_sum<3>(s, red);
    if (threadIdx.x == 0) {
        u[3 * p] = s[0];
        u[3 * p + 1] = s[1];
        u[3 * p + 2] = s[2];
    }
}

// One warp per row: c = C u (C row-major nc x nc; FP32 products and sums,
// the accuracy of the inner operator).
__global__ void k_coarse_gemv(int nc, const float* __restrict__ C, const double* __restrict__ u,
                              float* __restrict__ c) {
    const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= nc) return;
    const float* row = C + (int64_t)r * nc;
    float s = 0.0f;
    for (int k = lane; k < nc; k += 32) s = fmaf(row[k], (float)u[k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) c[r] = s;
}

// One block per target particle P: w_P -= sum over P's entries (P, Q) of
// W_e c_Q.
__global__ void __launch_bounds__(CO_TPB)
    k_coarse_prolong_w(int npp, const int* __restrict__ off, const int2* __restrict__ ent,
                       const float* __restrict__ W, const float* __restrict__ c,
                       double* __restrict__ w) {
    const int P = blockIdx.x;
    const int e0 = off[P], e1 = off[P + 1];
    const int64_t base = (int64_t)P * npp;
    for (int t = threadIdx.x; t < npp; t += CO_TPB) {
        float s = 0.0f;
        for (int e = e0; e < e1; ++e) {
            const int Q = ent[e].y;
            const float* We = W + (int64_t)e * 3 * npp;
            s = fmaf(We[t], c[3 * Q], s);
            s = fmaf(We[npp + t], c[3 * Q + 1], s);
            s = fmaf(We[2 * npp + t], c[3 * Q + 2], s);
        }
        w[base + t] -= (double)s;
    }
}

// s = sum_{k < k1} y_k U[k] (coarse vectors of length nc).
__global__ void k_coarse_combine(int nc, int k1, const double* __restrict__ U,
                                 const double* __restrict__ y, double* __restrict__ s) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nc) return;
    double a = 0.0;
    for (int k = 0; k < k1; ++k) a = fma(U[(int64_t)k * nc + r], y[k], a);
    s[r] = a;
}

// t -= Z c (Z: three vectors of length n, one column per particle each).
__global__ void k_coarse_prolong_z(int npp, int64_t n, const double* __restrict__ Z,
                                   const float* __restrict__ c, double* __restrict__ t) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = (int)(i / npp);
    t[i] -= Z[i] * c[3 * p] + Z[n + i] * c[3 * p + 1] + Z[2 * n + i] * c[3 * p + 2];
}

// ---------------------------------------------------------------------------
// Host side

static bool coarse_eligible(const yk_geom* g) {
    const yk_params& P = g->prm;
    return P.coarse == YK_COARSE_MODES && P.precision == YK_MIXED &&
           P.precond == YK_PRECOND_BLOCK && P.representation == YK_REP_DOUBLE_LAYER &&
           g->use_self && g->np >= 2 && g->np <= COARSE_MAX_PARTICLES;
}

// Device memory of the coarse space for a request (serving admission): the
// coupled pairs are estimated from the particle density over the centres'
// bounding box (twice the uniform-density count, at most np per particle).
size_t coarse_bytes(const yk_particle* parts, int np, const yk_params& P) {
    if (P.coarse != YK_COARSE_MODES || P.precision != YK_MIXED || P.precond != YK_PRECOND_BLOCK ||
        np < 2 || np > COARSE_MAX_PARTICLES)
        return 0;
    double rmax = 0.0, x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (int i = 0; i < np; ++i) {
        rmax = std::max(rmax, std::max(parts[i].A, parts[i].B));
        x0 = std::min(x0, parts[i].cx);
        x1 = std::max(x1, parts[i].cx);
        y0 = std::min(y0, parts[i].cy);
        y1 = std::max(y1, parts[i].cy);
    }
    const double gap = cutoff_gap(P.rho, 2.0 * PI * rmax, COARSE_TOL);
    const double area = (x1 - x0 + 2.0 * rmax) * (y1 - y0 + 2.0 * rmax);
    const double reach = gap + 2.0 * rmax;
    const double per = isfinite(reach) ? 1.0 + 2.0 * np * PI * reach * reach / area : (double)np;
    const size_t nent = (size_t)np * (size_t)std::min((double)np, per);
    const size_t npp = (size_t)P.n_panels * P.n_gl, nc = 3 * (size_t)np;
    if (nent * 3 * npp > COARSE_MAX_W_FLOATS) return 0;
    return nent * (3 * npp * sizeof(float) + sizeof(int2)) + nc * nc * sizeof(float) +
           9 * np * npp * sizeof(double) + ((size_t)P.gmres_restart + 2) * nc * sizeof(double) +
           (GJ_W * GJ_W + 2 * GJ_W * nc) * sizeof(float);
}

static int coarse_alloc(yk_geom* g) {
    Coarse& K = g->coarse;
    if (K.Z) return YK_OK;
    cudaStream_t st = g->ctx->stream;
    const int np = g->np, nc = 3 * np;
    const size_t n = (size_t)g->n;
    K.nc = nc;
    YK_TRY(dev_alloc((void**)&K.off, sizeof(int) * (np + 1), st));
    YK_TRY(dev_alloc((void**)&K.Z, sizeof(double) * 3 * n, st));
    YK_TRY(dev_alloc((void**)&K.Y, sizeof(double) * 3 * n, st));
    YK_TRY(dev_alloc((void**)&K.O, sizeof(double) * 3 * n, st));
    YK_TRY(dev_alloc((void**)&K.C, sizeof(float) * (size_t)nc * nc, st));
    YK_TRY(dev_alloc((void**)&K.piv, sizeof(float) * (GJ_W * GJ_W + 2 * (size_t)GJ_W * nc), st));
    YK_TRY(dev_alloc((void**)&K.U, sizeof(double) * (size_t)g->ws.m * nc, st));
    YK_TRY(dev_alloc((void**)&K.cv, sizeof(double) * 2 * (size_t)nc, st));
    YK_TRY(dev_alloc((void**)&K.flag, sizeof(int), st));
    return YK_OK;
}

int coarse_prepare(yk_geom* g) {
    Coarse& K = g->coarse;
    if (!coarse_eligible(g)) {
        K.on = false;
        return YK_OK;
    }
    if (K.valid) return YK_OK;
    K.on = false;
    // near-contact corrections act between particles outside the stored
    // couplings: no deflation for such configurations
    int ntgt = 0;
    YK_TRY(contact_targets(g, &ntgt));
    if (ntgt > 0) {
        K.valid = true;
        return YK_OK;
    }
    YK_TRY(coarse_alloc(g));
    cudaStream_t st = g->ctx->stream;
    const int np = g->np, npp = g->npp, nc = K.nc;
    const int64_t n = g->n;
    GeomView G = g->view();
    // coupled particle pairs
    const double gap = cutoff_gap(g->prm.rho, g->max_perimeter, COARSE_TOL);
    int* counts = (int*)g->ws.partial;   // np ints of scratch
    const int wblocks = ceil_div((int64_t)np * 32, CO_TPB);
    YK_LAUNCH(k_coarse_count, wblocks, CO_TPB, 0, st, np, g->d_part, gap, counts);
    YK_LAUNCH(k_coarse_scan, 1, 32, 0, st, np, counts, K.off);
    int nent = 0;
    YK_TRY_CUDA(cudaMemcpyAsync(&nent, K.off + np, sizeof(int), cudaMemcpyDeviceToHost, st));
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    if (nent > K.cap) {
        dev_free(K.ent, st);
        K.ent = nullptr;
        K.cap = 0;
        YK_TRY(dev_alloc((void**)&K.ent, sizeof(int2) * (size_t)nent, st));
        K.cap = nent;
    }
    const size_t wneed = (size_t)nent * 3 * npp;
    if (wneed > COARSE_MAX_W_FLOATS) {   // couplings too wide-reaching to store: no deflation
        K.valid = true;
        return YK_OK;
    }
    if (wneed > K.wcap) {
        dev_free(K.W, st);
        K.W = nullptr;
        K.wcap = 0;
        YK_TRY(dev_alloc((void**)&K.W, sizeof(float) * wneed, st));
        K.wcap = wneed;
    }
    YK_LAUNCH(k_coarse_fill, wblocks, CO_TPB, 0, st, np, g->d_part, gap, K.off, K.ent);
    // Z, Y = M Z, O = own part of A Y
    YK_LAUNCH(k_coarse_modes, np, CO_TPB, 0, st, G, K.Z);
    for (int c = 0; c < 3; ++c) {
        YK_TRY(apply_preconditioner(g, K.Z + c * n, K.Y + c * n, true));
        YK_TRY(own_apply_f32(g, K.Y + c * n, K.O + c * n));
    }
    // B Z and Z^T B Z
    YK_TRY_CUDA(cudaMemsetAsync(K.C, 0, sizeof(float) * (size_t)nc * nc, st));
    const float kpf = (float)(LOG2E / g->prm.rho);
    const float ks = (float)(sqrt(LOG2E) / (2.0 * PI * g->prm.rho));
    const size_t smem = sizeof(float4) * 2 * (size_t)npp;
    YK_LAUNCH(k_coarse_blocks, nent, CO_TPB, smem, st, G, K.ent, K.Y, K.O, K.Z, kpf, ks, K.W, K.C,
              nc);
    // (Z^T B Z)^{-1}
    YK_TRY_CUDA(cudaMemsetAsync(K.flag, 0, sizeof(int), st));
    float* Dinv = K.piv;
    float* Cp = K.piv + GJ_W * GJ_W;
    float* R = Cp + (size_t)nc * GJ_W;
    for (int k0 = 0; k0 < nc; k0 += GJ_W) {
        const int w = std::min(GJ_W, nc - k0);
        YK_LAUNCH(k_gj_pivot, 1, CO_TPB, 0, st, nc, k0, w, K.C, Dinv, K.flag);
        YK_LAUNCH(k_gj_panel, dim3(ceil_div(nc, GJ_PTPB), ceil_div(w, GJ_PROWS)), GJ_PTPB, 0, st,
                  nc, k0, w, K.C, Dinv, Cp, R);
        YK_LAUNCH(k_gj_update, dim3(ceil_div(nc, GJ_COLS), ceil_div(nc, GJ_ROWS)), GJ_COLS, 0, st,
                  nc, k0, w, K.C, Dinv, Cp, R);
    }
    int* hf = (int*)host_status(g->ctx);
    if (!hf) return YK_ERR_NO_MEMORY;
    YK_TRY_CUDA(cudaMemcpyAsync(hf, K.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    YK_TRY_CUDA(cudaGetLastError());
    K.valid = true;
    K.on = (*hf == 0);
    return YK_OK;
}

// w = A M v_j  ->  B P v_j = w - (B Z) C Z^T (w - v_j); keeps Z^T (w - v_j).
int coarse_deflate(yk_geom* g, const double* v, double* w, int j) {
    Coarse& K = g->coarse;
    cudaStream_t st = g->ctx->stream;
    double* u = K.U + (int64_t)j * K.nc;
    float* c = (float*)(K.cv + K.nc);
    YK_LAUNCH(k_coarse_restrict, g->np, CO_TPB, 0, st, g->npp, g->n, K.Z, w, v, u);
    YK_LAUNCH(k_coarse_gemv, ceil_div((int64_t)K.nc * 32, 256), 256, 0, st, K.nc, K.C, u, c);
    YK_LAUNCH(k_coarse_prolong_w, g->np, CO_TPB, 0, st, g->npp, K.off, K.ent, K.W, c, w);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

// The coarse term of a cycle's correction: M P V y = Z_kept y - (M Z) C
// sum_k y_k Z^T (B v_k - v_k); x -= Y C sum_k y_k u_k (Y = M Z).
int coarse_correct(yk_geom* g, int k, const double* y, double* x) {
    Coarse& K = g->coarse;
    cudaStream_t st = g->ctx->stream;
    double* s = K.cv;
    float* c = (float*)(K.cv + K.nc);
    YK_LAUNCH(k_coarse_combine, ceil_div(K.nc, 256), 256, 0, st, K.nc, k, K.U, y, s);
    YK_LAUNCH(k_coarse_gemv, ceil_div((int64_t)K.nc * 32, 256), 256, 0, st, K.nc, K.C, s, c);
    YK_LAUNCH(k_coarse_prolong_z, ceil_div(g->n, 256), 256, 0, st, g->npp, g->n, K.Y, c, x);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

void coarse_free(yk_geom* g) {
    Coarse& K = g->coarse;
    cudaStream_t st = g->ctx->stream;
    void* bufs[] = {K.off, K.ent, K.Z, K.Y, K.O, K.W, K.C, K.piv, K.U, K.cv, K.flag};
    for (void* b : bufs) dev_free(b, st);
    K = Coarse{};
}

}  // namespace yk
