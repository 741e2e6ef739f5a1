// Far-field (point-to-point) part of the double-layer operator and of its
// normal derivative, and the assembly y = far + near (Eq. bie with the QBX
// near rows of Section 5).
//
// Far kernel (Eq. double-layer-def with G = K0(r/rho)/2pi, Eq. Gfunc):
//   dG/dnu_y = K1(r/rho) ((x - y) . nu_y) / (2 pi rho r).
// Normal derivative at a boundary target with normal nu_x:
//   nu_x . grad_x dG/dnu_y = [g (nu_y . nu_x) + g'(r) (d . nu_y)(d . nu_x)/r] / 2pi,
//   g = K1(z)/(rho r), g' = -(K0(z)/rho + 2 K1(z)/r)/(rho r), z = r/rho, d = x - y.
//
// Work decomposition: blockIdx.x = 256 consecutive targets (one per thread),
// blockIdx.y = a chunk of consecutive source particles. Each source
// particle's nodes are staged in shared memory and swept by all targets;
// the per-chunk sums go to partial[chunk][target] and k_assemble adds the
// chunks in a fixed order (deterministic) plus the near rows.
// Sources that are the target's own near panels are skipped: the QBX rows
// replace them.
#include <math.h>

#include <algorithm>

#include "bessel.cuh"
#include "yk_internal.cuh"

namespace yk {

constexpr int TPB = 256;        // targets per block
constexpr int STILE = 256;      // source nodes staged per pass
constexpr float LOG2E_F = 1.4426950408889634f;

__device__ __forceinline__ bool is_near_panel(int pt_panel, int ps_panel, int npan, int w) {
    if (2 * w + 1 >= npan) return true;
    int d = ps_panel - pt_panel;
    d = ((d % npan) + npan) % npan;
    return d <= w || npan - d <= w;
}

// ---------------------------------------------------------------------------
// FP64 far field (value or normal derivative)
// ---------------------------------------------------------------------------
template <bool GRAD>
__global__ void __launch_bounds__(TPB) k_p2p_f64(GeomView G, const double* __restrict__ sigma,
                                                 int ppc, double* __restrict__ partial) {
    __shared__ yk::d4 src[STILE];
    const int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x;
    const bool active = i < G.n;
    const int64_t ii = active ? i : 0;
    const double tx = G.x[ii], ty = G.y[ii];
    const double tnx = GRAD ? G.nx[ii] : 0.0, tny = GRAD ? G.ny[ii] : 0.0;
    const int pt = (int)(ii / G.npp);
    const int tpan = (int)(ii % G.npp) / G.ngl;
    const double rho = G.rho, kappa = 1.0 / rho, two_rho = 2.0 * rho;
    const int s0 = blockIdx.y * ppc;
    const int s1 = min(G.np, s0 + ppc);
    double acc = 0.0;
    for (int s = s0; s < s1; ++s) {
        const int64_t base = (int64_t)s * G.npp;
        const bool own = (s == pt);
        for (int jb = 0; jb < G.npp; jb += STILE) {
            const int cnt = min(STILE, G.npp - jb);
            __syncthreads();
            if (threadIdx.x < cnt) {
                const int64_t j = base + jb + threadIdx.x;
                const double ws = G.w[j] * sigma[j];
                src[threadIdx.x] = make_d4(G.x[j], G.y[j], ws * G.nx[j], ws * G.ny[j]);
            }
            __syncthreads();
            if (!active) continue;
            for (int q = 0; q < cnt; ++q) {
                if (own && is_near_panel(tpan, (jb + q) / G.ngl, G.npan, G.near_w)) continue;
                const yk::d4 S = src[q];
                const double dx = tx - S.x, dy = ty - S.y;
                const double r2 = fma(dx, dx, dy * dy);
                const double ri = rsqrt(r2);
                const double z = r2 * ri * kappa;
                if (!GRAD) {
                    double k1v;
                    if (z <= 2.0) k1v = k1_series(z);
                    else k1v = exp(-z) * p1_large(two_rho * ri) * rsqrt(z);
                    acc = fma(k1v * ri, fma(dx, S.z, dy * S.w), acc);
                } else {
                    double k0v, k1v;
                    k01(z, k0v, k1v);
                    const double g = k1v * ri * kappa;
                    const double gp = -(k0v * kappa + 2.0 * k1v * ri) * kappa * ri;
                    const double dn_s = fma(dx, S.z, dy * S.w);     // (d . nu_y) w sigma
                    const double nn = fma(tnx, S.z, tny * S.w);     // (nu_x . nu_y) w sigma
                    const double dn_t = fma(dx, tnx, dy * tny);     // d . nu_x
                    acc += g * nn + gp * dn_s * dn_t * ri;
                }
            }
        }
    }
    if (active) {
        const double scale = GRAD ? 1.0 / (2.0 * PI) : 1.0 / (2.0 * PI * rho);
        partial[blockIdx.y * G.n + i] = acc * scale;
    }
}

// ---------------------------------------------------------------------------
// FP32 far field with FP64 accumulation (value only; the inner operator of
// the mixed solver). Coordinates are FP32 offsets from each particle's
// centre, pre-scaled by log2(e)/rho, so that exp(-r/rho) = exp2(-z') with
// z' = |d'| and t = 2/z = 2 log2(e)/z'. A target-source particle pair
// contributes through the FP64 centre difference rounded once to FP32.
// For z > 2: K1(z) = exp(-z) z^{-1/2} P(2t - 1), t = 2/z. Each thread owns
// two targets (tid and tid + 128) so that every staged source feeds two
// pairs. The special functions are the single-instruction approximations
// ex2.approx.ftz and rsqrt.approx.ftz (relative error ~2^-22).
// ---------------------------------------------------------------------------
constexpr int F32_TPB = 128;     // threads per block (2 targets each)

__device__ __forceinline__ float ex2_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_fast(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct PairF32 {
    // z > 2: exp2(-z') P(s) z'^{-1/2} (D'.g)/z' = K1(z) (D'.g) / (z' sqrt(log2 e))
    __device__ __forceinline__ static float far(float dX, float dY, float gx, float gy) {
        const float z2 = fmaf(dX, dX, dY * dY);
        const float rz = rsqrt_fast(z2);              // 1/z'
        const float zp = z2 * rz;                     // z' = z log2 e
        const float s = fmaf(4.0f * LOG2E_F, rz, -1.0f);   // 2t - 1
        const float P = hornerf(YK_P1_F32, s);
        const float e = ex2_fast(-zp);
        const float sq = rsqrt_fast(zp);              // (z log2 e)^{-1/2}
        return (e * P * sq) * (rz * fmaf(dX, gx, dY * gy));
    }
    // general pair (any z), same units as far(): K1(z) (D'.g) / (z' sqrt(log2 e))
    __device__ __forceinline__ static float any(float dX, float dY, float gx, float gy) {
        const float z2 = fmaf(dX, dX, dY * dY);
        const float rz = rsqrt_fast(z2);
        const float zp = z2 * rz;
        const float z = zp * (1.0f / LOG2E_F);
        if (z > 2.0f) return far(dX, dY, gx, gy);
        const float k1v = k1f(z, 2.0f / z);
        return k1v * rsqrtf(LOG2E_F) * (rz * fmaf(dX, gx, dY * gy));
    }
};

struct TargetF32 {
    float TX, TY;       // scaled target position relative to the source particle
    bool close, own;
    int pan;
};

__device__ __forceinline__ void sweep_general(const float4* src, int jb, int cnt, const GeomView& G,
                                              const TargetF32& T, float& acc) {
    for (int q = 0; q < cnt; ++q) {
        if (T.own && is_near_panel(T.pan, (jb + q) / G.ngl, G.npan, G.near_w)) continue;
        const float4 S = src[q];
        acc += PairF32::any(T.TX - S.x, T.TY - S.y, S.z, S.w);
    }
}

__global__ void __launch_bounds__(F32_TPB) k_p2p_f32(GeomView G, const double* __restrict__ sigma,
                                                     int ppc, float kscale,
                                                     double* __restrict__ partial) {
    __shared__ float4 src[STILE];
    const int64_t i0 = blockIdx.x * (int64_t)TPB + threadIdx.x;
    const int64_t i1 = i0 + F32_TPB;
    const bool act0 = i0 < G.n, act1 = i1 < G.n;
    const int64_t ii0 = act0 ? i0 : 0, ii1 = act1 ? i1 : 0;
    const float2 xi0 = G.xi[ii0], xi1 = G.xi[ii1];
    const int pt0 = (int)(ii0 / G.npp), pt1 = (int)(ii1 / G.npp);
    const int pan0 = (int)(ii0 % G.npp) / G.ngl, pan1 = (int)(ii1 % G.npp) / G.ngl;
    const yk::d4 at0 = G.part[pt0], at1 = G.part[pt1];
    const double kp = 1.4426950408889634 / G.rho;   // log2(e) / rho
    const float kpf = (float)kp;
    const double near_gap = 2.0 * G.rho;            // below this a pair may have z <= 2
    const int s0 = blockIdx.y * ppc;
    const int s1 = min(G.np, s0 + ppc);
    double acc0 = 0.0, acc1 = 0.0;
    for (int s = s0; s < s1; ++s) {
        const int64_t base = (int64_t)s * G.npp;
        const yk::d4 as = G.part[s];
        TargetF32 T0, T1;
        {
            const double dx = at0.x - as.x, dy = at0.y - as.y;
            T0.own = (s == pt0);
            T0.close = T0.own || (sqrt(dx * dx + dy * dy) - at0.z - as.z <= near_gap);
            T0.TX = (float)(kp * dx) + kpf * xi0.x;
            T0.TY = (float)(kp * dy) + kpf * xi0.y;
            T0.pan = pan0;
        }
        {
            const double dx = at1.x - as.x, dy = at1.y - as.y;
            T1.own = (s == pt1);
            T1.close = T1.own || (sqrt(dx * dx + dy * dy) - at1.z - as.z <= near_gap);
            T1.TX = (float)(kp * dx) + kpf * xi1.x;
            T1.TY = (float)(kp * dy) + kpf * xi1.y;
            T1.pan = pan1;
        }
        for (int jb = 0; jb < G.npp; jb += STILE) {
            const int cnt = min(STILE, G.npp - jb);
            __syncthreads();
            for (int q = threadIdx.x; q < cnt; q += F32_TPB) {
                const int64_t j = base + jb + q;
                const float2 xs = G.xi[j];
                const double ws = G.w[j] * sigma[j];
                src[q] = make_float4(kpf * xs.x, kpf * xs.y, (float)(ws * G.nx[j]),
                                     (float)(ws * G.ny[j]));
            }
            __syncthreads();
            float a0 = 0.0f, b0 = 0.0f, a1 = 0.0f, b1 = 0.0f;
            if (!T0.close && !T1.close) {
                int q = 0;
#pragma unroll 2
                for (; q + 2 <= cnt; q += 2) {
                    const float4 S = src[q], U = src[q + 1];
                    a0 += PairF32::far(T0.TX - S.x, T0.TY - S.y, S.z, S.w);
                    a1 += PairF32::far(T1.TX - S.x, T1.TY - S.y, S.z, S.w);
                    b0 += PairF32::far(T0.TX - U.x, T0.TY - U.y, U.z, U.w);
                    b1 += PairF32::far(T1.TX - U.x, T1.TY - U.y, U.z, U.w);
                }
                if (q < cnt) {
                    const float4 S = src[q];
                    a0 += PairF32::far(T0.TX - S.x, T0.TY - S.y, S.z, S.w);
                    a1 += PairF32::far(T1.TX - S.x, T1.TY - S.y, S.z, S.w);
                }
            } else {
                sweep_general(src, jb, cnt, G, T0, a0);
                sweep_general(src, jb, cnt, G, T1, a1);
            }
            acc0 += (double)(a0 + b0);
            acc1 += (double)(a1 + b1);
        }
    }
    if (act0) partial[blockIdx.y * G.n + i0] = acc0 * (double)kscale;
    if (act1) partial[blockIdx.y * G.n + i1] = acc1 * (double)kscale;
}

// ---------------------------------------------------------------------------
// Precision-split far field (value or normal derivative): a source particle
// whose FP32 error bound is below the split tolerance (its gap to the
// target's particle is at least split_gap) is swept in FP32; closer ones
// in FP64. Used for the FP64-accurate residual and gradient of the mixed
// solver.
// ---------------------------------------------------------------------------
template <bool GRAD>
__global__ void __launch_bounds__(TPB) k_p2p_split(GeomView G, const double* __restrict__ sigma,
                                                   int ppc, double split_gap,
                                                   double* __restrict__ partial) {
    __shared__ yk::d4 src[STILE];
    __shared__ float4 srcf[STILE];
    const int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x;
    const bool active = i < G.n;
    const int64_t ii = active ? i : 0;
    const double tx = G.x[ii], ty = G.y[ii];
    const double tnx = GRAD ? G.nx[ii] : 0.0, tny = GRAD ? G.ny[ii] : 0.0;
    const float2 xit = G.xi[ii];
    const int pt = (int)(ii / G.npp);
    const int tpan = (int)(ii % G.npp) / G.ngl;
    const yk::d4 at = G.part[pt];
    const double rho = G.rho, kappa = 1.0 / rho, two_rho = 2.0 * rho;
    const float rhof = (float)rho, kappaf = (float)kappa;
    const int s0 = blockIdx.y * ppc;
    const int s1 = min(G.np, s0 + ppc);
    double acc = 0.0;
    for (int s = s0; s < s1; ++s) {
        const int64_t base = (int64_t)s * G.npp;
        const yk::d4 as = G.part[s];
        const bool own = (s == pt);
        const double ddx = at.x - as.x, ddy = at.y - as.y;
        const bool use64 = own || (sqrt(ddx * ddx + ddy * ddy) - at.z - as.z < split_gap);
        // block-uniform staging of both forms; each thread sweeps one
        const float TX = (float)ddx + xit.x, TY = (float)ddy + xit.y;
        for (int jb = 0; jb < G.npp; jb += STILE) {
            const int cnt = min(STILE, G.npp - jb);
            __syncthreads();
            if (threadIdx.x < cnt) {
                const int64_t j = base + jb + threadIdx.x;
                const double ws = G.w[j] * sigma[j];
                const double gx = ws * G.nx[j], gy = ws * G.ny[j];
                src[threadIdx.x] = make_d4(G.x[j], G.y[j], gx, gy);
                const float2 xs = G.xi[j];
                srcf[threadIdx.x] = make_float4(xs.x, xs.y, (float)gx, (float)gy);
            }
            __syncthreads();
            if (!active) continue;
            if (use64) {
                for (int q = 0; q < cnt; ++q) {
                    if (own && is_near_panel(tpan, (jb + q) / G.ngl, G.npan, G.near_w)) continue;
                    const yk::d4 S = src[q];
                    const double dx = tx - S.x, dy = ty - S.y;
                    const double r2 = fma(dx, dx, dy * dy);
                    const double ri = rsqrt(r2);
                    const double z = r2 * ri * kappa;
                    if (!GRAD) {
                        double k1v;
                        if (z <= 2.0) k1v = k1_series(z);
                        else k1v = exp(-z) * p1_large(two_rho * ri) * rsqrt(z);
                        acc = fma(k1v * ri * kappa, fma(dx, S.z, dy * S.w), acc);
                    } else {
                        double k0v, k1v;
                        k01(z, k0v, k1v);
                        const double g = k1v * ri * kappa;
                        const double gp = -(k0v * kappa + 2.0 * k1v * ri) * kappa * ri;
                        const double dn_s = fma(dx, S.z, dy * S.w);
                        const double nn = fma(tnx, S.z, tny * S.w);
                        const double dn_t = fma(dx, tnx, dy * tny);
                        acc += g * nn + gp * dn_s * dn_t * ri;
                    }
                }
            } else {
                float a0 = 0.0f, a1 = 0.0f;
                const float tnxf = (float)tnx, tnyf = (float)tny;
                for (int q = 0; q < cnt; ++q) {
                    const float4 S = srcf[q];
                    const float dx = TX - S.x, dy = TY - S.y;
                    const float r2 = fmaf(dx, dx, dy * dy);
                    const float ri = rsqrtf(r2);
                    const float z = r2 * ri * kappaf;
                    const float t = 2.0f * rhof * ri;
                    if (!GRAD) {
                        const float k1v = k1f(z, t);
                        const float v = k1v * ri * kappaf * fmaf(dx, S.z, dy * S.w);
                        if (q & 1) a1 += v; else a0 += v;
                    } else {
                        float k0v, k1v;
                        k01f(z, t, k0v, k1v);
                        const float g = k1v * ri * kappaf;
                        const float gp = -(k0v * kappaf + 2.0f * k1v * ri) * kappaf * ri;
                        const float dn_s = fmaf(dx, S.z, dy * S.w);
                        const float nn = fmaf(tnxf, S.z, tnyf * S.w);
                        const float dn_t = fmaf(dx, tnxf, dy * tnyf);
                        const float v = g * nn + gp * dn_s * dn_t * ri;
                        if (q & 1) a1 += v; else a0 += v;
                    }
                }
                acc += (double)(a0 + a1);
            }
        }
    }
    if (active) partial[blockIdx.y * G.n + i] = acc * (1.0 / (2.0 * PI));
}

// y_i = sum_chunks partial[c][i] + sum_near C[shape][local i][c] sigma[near c]
__global__ void k_assemble(GeomView G, int nchunk, const double* __restrict__ partial,
                           const double* __restrict__ rows, const double* __restrict__ sigma,
                           double* __restrict__ y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= G.n) return;
    double acc = 0.0;
    for (int c = 0; c < nchunk; ++c) acc += partial[c * G.n + i];
    const int p = (int)(i / G.npp);
    const int li = (int)(i % G.npp);
    const int k = li / G.ngl;
    const int rowlen = G.n_near * G.ngl;
    const double* row = rows + ((int64_t)G.shape_of[p] * G.npp + li) * rowlen;
    const int64_t base = (int64_t)p * G.npp;
    double nr = 0.0;
    for (int q = 0; q < G.n_near; ++q) {
        const int pk = (2 * G.near_w + 1 >= G.npan) ? q
                       : ((k - G.near_w + q) % G.npan + G.npan) % G.npan;
        const double* sq = sigma + base + (int64_t)pk * G.ngl;
        const double* rq = row + q * G.ngl;
        for (int j = 0; j < G.ngl; ++j) nr = fma(rq[j], sq[j], nr);
    }
    y[i] = acc + nr;
}

// u(t) = D[sigma](t) at off-surface targets, FP64, all sources.
__global__ void __launch_bounds__(TPB) k_potential(GeomView G, const double* __restrict__ sigma,
                                                   const double* __restrict__ tgt, int64_t nt,
                                                   int ppc, double* __restrict__ partial) {
    __shared__ yk::d4 src[STILE];
    const int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x;
    const bool active = i < nt;
    const double tx = active ? tgt[2 * i] : 0.0, ty = active ? tgt[2 * i + 1] : 0.0;
    const double rho = G.rho, kappa = 1.0 / rho, two_rho = 2.0 * rho;
    const int s0 = blockIdx.y * ppc;
    const int s1 = min(G.np, s0 + ppc);
    double acc = 0.0;
    for (int s = s0; s < s1; ++s) {
        const int64_t base = (int64_t)s * G.npp;
        for (int jb = 0; jb < G.npp; jb += STILE) {
            const int cnt = min(STILE, G.npp - jb);
            __syncthreads();
            if (threadIdx.x < cnt) {
                const int64_t j = base + jb + threadIdx.x;
                const double ws = G.w[j] * sigma[j];
                src[threadIdx.x] = make_d4(G.x[j], G.y[j], ws * G.nx[j], ws * G.ny[j]);
            }
            __syncthreads();
            if (!active) continue;
            for (int q = 0; q < cnt; ++q) {
                const yk::d4 S = src[q];
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

__global__ void k_sum_chunks(int64_t n, int nchunk, const double* __restrict__ partial,
                             double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int c = 0; c < nchunk; ++c) acc += partial[c * n + i];
    out[i] = acc;
}

// ---------------------------------------------------------------------------
static int chunking(const yk_geom* g, int* ppc) {
    const int nct = ceil_div(g->n, TPB);
    int nchunk = g->ws.nchunk;
    *ppc = ceil_div(g->np, nchunk);
    (void)nct;
    return ceil_div(g->np, *ppc);
}

int matvec(yk_geom* g, const double* sigma, double* y, Prec prec) {
    cudaStream_t st = g->ctx->stream;
    GeomView G = g->view();
    int ppc;
    const int nchunk = chunking(g, &ppc);
    dim3 grid(ceil_div(g->n, TPB), nchunk);
    if (prec == Prec::F64) {
        YK_LAUNCH(k_p2p_f64<false>, grid, TPB, 0, st, G, sigma, ppc, g->ws.partial);
    } else if (prec == Prec::F32) {
        // PairF32 returns K1(z) (d . g)/r / sqrt(log2 e) in scaled units
        const double ks = sqrt(1.4426950408889634) / (2.0 * PI * g->prm.rho);
        YK_LAUNCH(k_p2p_f32, grid, F32_TPB, 0, st, G, sigma, ppc, (float)ks, g->ws.partial);
    } else {
        YK_LAUNCH(k_p2p_split<false>, grid, TPB, 0, st, G, sigma, ppc, g->split_gap, g->ws.partial);
    }
    YK_LAUNCH(k_assemble, ceil_div(g->n, 256), 256, 0, st, G, nchunk, g->ws.partial, G.cval, sigma, y);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

int normal_derivative(yk_geom* g, const double* sigma, double* un, Prec prec) {
    cudaStream_t st = g->ctx->stream;
    GeomView G = g->view();
    int ppc;
    const int nchunk = chunking(g, &ppc);
    dim3 grid(ceil_div(g->n, TPB), nchunk);
    if (prec == Prec::F64) {
        YK_LAUNCH(k_p2p_f64<true>, grid, TPB, 0, st, G, sigma, ppc, g->ws.partial);
    } else {
        YK_LAUNCH(k_p2p_split<true>, grid, TPB, 0, st, G, sigma, ppc, g->split_gap_grad,
                  g->ws.partial);
    }
    YK_LAUNCH(k_assemble, ceil_div(g->n, 256), 256, 0, st, G, nchunk, g->ws.partial, G.cgrad, sigma, un);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

int potential(yk_geom* g, const double* sigma, const double* targets, int64_t nt, double* u) {
    if (nt <= 0) return YK_OK;
    cudaStream_t st = g->ctx->stream;
    GeomView G = g->view();
    const int nct = ceil_div(nt, TPB);
    int nchunk = std::max(1, std::min(g->np, ceil_div(4 * 152, nct)));
    const int ppc = ceil_div(g->np, nchunk);
    nchunk = ceil_div(g->np, ppc);
    double* part = nullptr;
    YK_TRY_CUDA(cudaMallocAsync((void**)&part, sizeof(double) * nchunk * nt, st));
    dim3 grid(nct, nchunk);
    YK_LAUNCH(k_potential, grid, TPB, 0, st, G, sigma, targets, nt, ppc, part);
    YK_LAUNCH(k_sum_chunks, ceil_div(nt, 256), 256, 0, st, nt, nchunk, part, u);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(part, st);
    YK_TRY_CUDA(e);
    return YK_OK;
}

}  // namespace yk
