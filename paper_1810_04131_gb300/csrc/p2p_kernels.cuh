// Device code of the far-field evaluators (included by p2p.cu, which holds
// the host side).
//
// Far-field (point-to-point) part of the double-layer operator and of its
// normal derivative, and the assembly y = far + near (Eq. bie with the QBX
// near rows of Section 5).
//
// Far kernel (Eq. double-layer-def with G = K0(r/rho)/2pi, Eq. Gfunc):
//   dG/dnu_y = K1(r/rho) ((x - y) . nu_y) / (2 pi rho r).
// Normal derivative at a boundary target with normal nu_x:
//   nu_x . grad_x dG/dnu_y = [g (nu_y . nu_x) + g'(r) (d . nu_y)(d . nu_x)/r] / 2pi,
//   g = K1(z)/(rho r), g' = -(K0(z)/rho + 2 K1(z)/r)/(rho r), z = r/rho, d = x - y.
// Sources that are the target's own near panels are skipped: the QBX rows
// replace them.
//
// The kernels:
//  * k_src_pairs: the pair-packed FP32 source records of the density, once
//    per operator application (read by every block of the FP32 kernels).
//  * k_p2p_f32: FP32 evaluation with FP64 accumulation per source particle
//    (systems without self blocks); blockIdx.x = 256 consecutive targets (two
//    per thread), blockIdx.y = a chunk of source particles, partial sums per
//    chunk. Per block and source particle, the range of node-pair distances
//    picks the evaluation: none (every pair underflows to an exact FP32
//    zero), the full or the short K1 fit, or an expansion about the
//    particle's 1/z'.
//  * k_p2p_f32_sym / k_p2p_f32_symg: the symmetric FP32 far field over a list
//    of particle pairs, value and normal derivative: one evaluation per node
//    pair serves both directions. With a skip distance the lists leave out
//    the particle pairs that the FP64 tiles handle (same FP64 predicate in
//    both places).
//  * k_p2p_f32_cut / k_p2p_f32_grad_cut: the same per target particle over
//    a neighbour list (cut-off and FMM near fields).
//  * k_tiles_f64<GRAD>: one block per listed particle pair (P, Q), P <= Q,
//    all in FP64. The pair kernels are symmetric in (i, j) up to the sign of
//    d (value) or exactly (gradient), so each kernel evaluation feeds both
//    targets: P's nodes through registers, Q's through a warp reduction and
//    shared-memory atomics. Results go to a FP64 buffer with atomics.
//  * k_assemble: chunk partials (fixed order) + FP64 tile sums + near rows.
//
// The __global__ kernels are compiled only where YK_DEFINE_P2P_KERNELS is
// defined (p2p.cu); other translation units (batch.cu) include this header
// for the device functions and constants alone.
#pragma once
#include <math.h>

#include "bessel.cuh"
#include "block_apply.cuh"
#include "geom_view.cuh"

namespace yk {


constexpr int TPB = 256;         // targets per far-field block
constexpr int STILE = 256;       // source nodes staged per pass
constexpr int F32_TPB = 128;     // FP32 kernels: two targets per thread
constexpr int TILE_TPB = 256;    // FP64 pair tiles
constexpr float LOG2E_F = 1.4426950408889634f;
constexpr float Z_SHORT = 10.0f;   // z at or above which the short FP32 fit applies
constexpr float ZP_ZERO = 128.0f;  // z' = z log2 e at or above which exp2(-z') flushes to 0
constexpr double LOG2E = 1.4426950408889634;

__device__ __forceinline__ bool is_near_panel(int pt_panel, int ps_panel, int npan, int w) {
    if (2 * w + 1 >= npan) return true;
    int d = ps_panel - pt_panel;
    d = ((d % npan) + npan) % npan;
    return d <= w || npan - d <= w;
}

// The particle-pair predicate "handled by the FP64 tiles": the same particle,
// or bounding circles closer than thr. Evaluated with explicitly rounded
// operations so that the list builder and the FP32 kernels agree bitwise.
__device__ __forceinline__ bool pair_in_tiles(const d4& a, const d4& b, double thr) {
    const double dx = __dsub_rn(a.x, b.x), dy = __dsub_rn(a.y, b.y);
    const double s = __dadd_rn(__dadd_rn(a.z, b.z), thr);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) < __dmul_rn(s, s);
}

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

// ---------------------------------------------------------------------------
// FP32 pair evaluation. Coordinates are FP32 offsets from each particle's
// centre, pre-scaled by log2(e)/rho, so that exp(-r/rho) = exp2(-z') with
// z' = |d'|, and t = 2/z = 2 log2(e)/z'. For z > 2:
// K1(z) = exp(-z) z^{-1/2} P1(2t - 1). The special functions are the
// single-instruction approximations ex2.approx.ftz and rsqrt.approx.ftz
// (relative error ~2^-22).
// ---------------------------------------------------------------------------
struct PairF32 {
    // z > 2: exp2(-z') P1(s) z'^{-1/2} (D'.g)/z' = K1(z) (D'.g) / (z' sqrt(log2 e))
    __device__ __forceinline__ static float far(float dX, float dY, float gx, float gy) {
        const float z2 = fmaf(dX, dX, dY * dY);
        const float rz = rsqrt_fast(z2);                     // 1/z'
        const float zp = z2 * rz;                            // z' = z log2 e
        const float s = fmaf(4.0f * LOG2E_F, rz, -1.0f);     // 2t - 1
        const float P = hornerf(YK_P1_F32, s);
        const float e = ex2_fast(-zp);
        const float sq = rsqrt_fast(zp);                     // (z log2 e)^{-1/2}
        return (e * P * sq) * (rz * fmaf(dX, gx, dY * gy));
    }
    // any z, same units as far()
    __device__ __forceinline__ static float any(float dX, float dY, float gx, float gy) {
        const float z2 = fmaf(dX, dX, dY * dY);
        const float rz = rsqrt_fast(z2);
        const float zp = z2 * rz;
        const float z = zp * (1.0f / LOG2E_F);
        if (z > 2.0f) return far(dX, dY, gx, gy);
        const float k1v = k1f(z, 2.0f / z);
        return k1v * rsqrtf(LOG2E_F) * (rz * fmaf(dX, gx, dY * gy));
    }
    // normal derivative, unscaled coordinates d = x - y, target normal (nx, ny):
    // [g (nu_x . G) + g' (d . G)(d . nu_x)/r] with G = w sigma nu_y (2 pi left out)
    __device__ __forceinline__ static float grad(float dx, float dy, float nx, float ny, float gx,
                                                 float gy, float kappa, float rho) {
        const float r2 = fmaf(dx, dx, dy * dy);
        const float ri = rsqrt_fast(r2);
        const float z = r2 * ri * kappa;
        const float t = 2.0f * rho * ri;
        float k0v, k1v;
        if (z > 2.0f) {
            const float e = ex2_fast(-z * LOG2E_F) * rsqrt_fast(z);
            const float s = 2.0f * t - 1.0f;
            k0v = e * hornerf(YK_P0_F32, s);
            k1v = e * hornerf(YK_P1_F32, s);
        } else {
            k01f(z, t, k0v, k1v);
        }
        const float g = k1v * ri * kappa;
        const float gp = -(k0v * kappa + 2.0f * k1v * ri) * kappa * ri;
        const float dn_s = fmaf(dx, gx, dy * gy);
        const float nn = fmaf(nx, gx, ny * gy);
        const float dn_t = fmaf(dx, nx, dy * ny);
        return fmaf(g, nn, gp * dn_s * dn_t * ri);
    }
};

struct TargetF32 {
    float TX, TY;       // (scaled) target position relative to the source particle's centre
    bool close, own, skip;
    int pan;
};

// Target-side set-up against source particle s (all in FP32 from the hi/lo
// centres, plus the FP64 tile predicate when a skip distance is given).
__device__ __forceinline__ void target_setup(TargetF32& T, const GeomView& G, int pt, int s,
                                             float2 xit, float scale, float near_gap,
                                             bool mask, double skip_gap, int pan) {
    const float4 ct = G.c32[pt], cs = G.c32[s];
    const float dX = (ct.x - cs.x) + (ct.z - cs.z);
    const float dY = (ct.y - cs.y) + (ct.w - cs.w);
    T.own = (s == pt);
    const float gap = sqrtf(dX * dX + dY * dY) - G.r32[pt] - G.r32[s];
    T.close = T.own || gap <= near_gap;
    T.skip = mask && pair_in_tiles(G.part[pt], G.part[s], skip_gap);
    T.TX = fmaf(scale, dX, scale * xit.x);
    T.TY = fmaf(scale, dY, scale * xit.y);
    T.pan = pan;
}

// Smallest bounding-circle gap, and largest centre distance plus both radii,
// between target particles [pa, pb] and source particle s, in FP32 from the
// hi/lo centres: every node pair's distance lies in [gap, far]. Every thread
// of a block that passes the same arguments gets the same values, so
// decisions taken on them are block-uniform.
struct PairRange {
    float gap, far;
};
__device__ __forceinline__ PairRange block_range(const GeomView& G, int pa, int pb, int s) {
    const float4 cs = G.c32[s];
    const float rs = G.r32[s];
    PairRange r{3.0e38f, 0.0f};
    for (int p = pa; p <= pb; ++p) {
        const float4 ct = G.c32[p];
        const float dX = (ct.x - cs.x) + (ct.z - cs.z);
        const float dY = (ct.y - cs.y) + (ct.w - cs.w);
        const float d = sqrtf(dX * dX + dY * dY), rsum = G.r32[p] + rs;
        r.gap = fminf(r.gap, d - rsum);
        r.far = fmaxf(r.far, d + rsum);
    }
    return r;
}

// Packed FP32 evaluation of two far pairs at once (one target, two sources)
// with the f32x2 FMA/ADD/MUL instructions of sm_100+: lanes .x/.y are the
// two sources. Sources are staged as pairs: A = (-X0, -X1, -Y0, -Y1) in
// scaled coordinates, B = (gx0, gx1, gy0, gy1). Returns the two terms in the
// units of PairF32::far (K1(z) (D'.g) / (z' sqrt(log2 e))) added to acc.
// NC = 7 evaluates the fit of P1 for every z > 2, NC = 4 the short fit,
// valid for z >= 9.5 (both within 1.5e-7 relative), NC = NARROW or NARROW3
// the expansion about the source particle's 1/z' (two MUFU operations a pair
// instead of three).
//
// Two source-particle classes, decided per block from the bounding-circle
// gap between the block's target particles and the source particle (the
// same FP32 arithmetic in every thread, hence block-uniform):
//  * gap >= Z_SHORT rho: the short fit (three FMA fewer per pair);
//  * gap >= ZP_ZERO / kappa' (z' >= 128 for every pair): exp2(-z') is below
//    2^-127, which ex2.approx.ftz flushes to +0, so every pair adds exactly
//    zero to the FP32 sum; the source particle is skipped, with a result
//    identical to evaluating it.

// Coefficients of one source particle's evaluation, each in both lanes of a
// float2, picked at run time so that all modes use the same registers:
//  * FIT_LONG: the fit of P1 for every z > 2 (7 terms);
//  * FIT_SHORT: the short fit (the first 4 of c);
//  * NARROW: every pair has 1/z' within a factor 1 +- eps of rc (eps <=
//    EPS_NARROW). Then g(rz) = rz^{1/2} P1(rz), with P1 the short fit
//    sum_j p_j rz^j, is sum_k a_k u^k with u = rz/rc - 1 and
//    a_k = sum_j p_j rc^{j+1/2} binom(j + 1/2, k), cut after k = 4 (the
//    binomial series of (1 + u)^{j+1/2}; the first term left out is below
//    0.03 eps^5 = 5e-8 relative). c[0..4] = a_k, c[5] = 1/rc, c[6] = -1.
//    This replaces the z'^{-1/2} MUFU operation with one FMA;
//  * NARROW3: the same, cut after k = 3 for eps <= EPS_NARROW3 (the first
//    term left out is below 0.04 eps^4 = 3e-8 relative), c[4] unused.
constexpr int FIT_LONG = 7, FIT_SHORT = 4, NARROW = 5, NARROW3 = 6;
constexpr float EPS_NARROW = 0.07f;
constexpr float EPS_NARROW3 = 0.03f;

__host__ __device__ constexpr float binom_half(int j, int k) {   // binom(j + 1/2, k)
    float b = 1.0f;
    for (int i = 0; i < k; ++i) b = b * ((float)j + 0.5f - (float)i) / (float)(i + 1);
    return b;
}

struct PolyRZ {
    float2 c[FIT_LONG];
    __device__ __forceinline__ PolyRZ(int mode, float rc) {
        if (mode == NARROW || mode == NARROW3) {
            const float sr = sqrtf(rc);
            float pj[FIT_SHORT];
            float pw = sr;
#pragma unroll
            for (int j = 0; j < FIT_SHORT; ++j) {
                pj[j] = YK_P1_F32_RZ[FIT_LONG + j] * pw;   // p_j rc^{j+1/2}
                pw *= rc;
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                float a = 0.0f;
#pragma unroll
                for (int j = FIT_SHORT - 1; j >= 0; --j) a = fmaf(pj[j], binom_half(j, k), a);
                c[k] = make_float2(a, a);
            }
            const float ir = 1.0f / rc;
            c[5] = make_float2(ir, ir);
            c[6] = make_float2(-1.0f, -1.0f);
            return;
        }
        const int off = (mode == FIT_SHORT) ? FIT_LONG : 0;
#pragma unroll
        for (int k = 0; k < FIT_LONG; ++k) {
            const float v = YK_P1_F32_RZ[min(off + k, FIT_LONG + FIT_SHORT - 1)];
            c[k] = make_float2(v, v);
        }
    }
};
static_assert(sizeof(YK_P1_F32_RZ) == (FIT_LONG + FIT_SHORT) * sizeof(float), "fit lengths");

// The mode of a source particle from its pair range (block-uniform).
__device__ __forceinline__ int far_mode(const PairRange& r, float short_gap, float kpf, float& rc) {
    rc = 0.0f;
    if (!(r.gap >= short_gap)) return FIT_LONG;
    const float lo = 1.0f / (kpf * r.far), hi = 1.0f / (kpf * r.gap);   // range of 1/z'
    if (hi - lo <= EPS_NARROW * (hi + lo)) {
        rc = 0.5f * (hi + lo);
        return (hi - lo <= EPS_NARROW3 * (hi + lo)) ? NARROW3 : NARROW;
    }
    return FIT_SHORT;
}

template <int NC>
__device__ __forceinline__ float2 far2(float2 TX, float2 TY, const float4& A, const float4& B,
                                       const PolyRZ& P, float2 acc) {
    const float2 dX = __fadd2_rn(TX, make_float2(A.x, A.y));
    const float2 dY = __fadd2_rn(TY, make_float2(A.z, A.w));
    const float2 z2 = __ffma2_rn(dX, dX, __fmul2_rn(dY, dY));
    const float2 rz = make_float2(rsqrt_fast(z2.x), rsqrt_fast(z2.y));   // 1/z'
    const float2 zp = __fmul2_rn(z2, rz);                                 // z'
    if constexpr (NC == NARROW || NC == NARROW3) {
        const float2 u = __ffma2_rn(rz, P.c[5], P.c[6]);                  // rz/rc - 1
        constexpr int top = (NC == NARROW) ? 4 : 3;
        float2 q = P.c[top];
#pragma unroll
        for (int k = top - 1; k >= 0; --k) q = __ffma2_rn(q, u, P.c[k]); // rz^{1/2} P1(rz)
        const float2 e = make_float2(ex2_fast(-zp.x), ex2_fast(-zp.y));
        const float2 dot = __ffma2_rn(dX, make_float2(B.x, B.y), __fmul2_rn(dY, make_float2(B.z, B.w)));
        return __ffma2_rn(__fmul2_rn(e, q), __fmul2_rn(rz, dot), acc);
    }
    float2 p = P.c[NC - 1];
#pragma unroll
    for (int k = NC - 2; k >= 0; --k) p = __ffma2_rn(p, rz, P.c[k]);     // P1 in rz
    const float2 e = make_float2(ex2_fast(-zp.x), ex2_fast(-zp.y));
    const float2 sq = make_float2(rsqrt_fast(zp.x), rsqrt_fast(zp.y));   // z'^{-1/2}
    const float2 dot = __ffma2_rn(dX, make_float2(B.x, B.y), __fmul2_rn(dY, make_float2(B.z, B.w)));
    return __ffma2_rn(__fmul2_rn(__fmul2_rn(e, p), sq), __fmul2_rn(rz, dot), acc);
}

// Scalar view of source q in the pair-packed staging.
__device__ __forceinline__ float4 src_scalar(const float4* A, const float4* B, int q) {
    const float4 a = A[q >> 1], b = B[q >> 1];
    return (q & 1) ? make_float4(-a.y, -a.w, b.y, b.w) : make_float4(-a.x, -a.z, b.x, b.z);
}

// Two pairs of a close (non-own) source particle: the packed far form,
// except that a lane with z <= 2 (z'^2 <= (2 log2 e)^2, outside the fitted
// polynomial's range) takes the series of PairF32::any instead.
constexpr float ZCUT2 = 4.0f * LOG2E_F * LOG2E_F;
__device__ __forceinline__ float2 close2(float2 TX, float2 TY, const float4& A, const float4& B,
                                         const PolyRZ& P, float2 acc) {
    const float2 dX = __fadd2_rn(TX, make_float2(A.x, A.y));
    const float2 dY = __fadd2_rn(TY, make_float2(A.z, A.w));
    const float z2x = fmaf(dX.x, dX.x, dY.x * dY.x), z2y = fmaf(dX.y, dX.y, dY.y * dY.y);
    if (z2x > ZCUT2 && z2y > ZCUT2) return far2<FIT_LONG>(TX, TY, A, B, P, acc);
    acc.x += PairF32::any(dX.x, dY.x, B.x, B.z);
    acc.y += PairF32::any(dX.y, dY.y, B.y, B.w);
    return acc;
}

// Packed FP32 normal derivative of two far pairs (one target with normal
// (nx, ny), two sources), same scaled coordinates and staging as far2. With
// E = exp2(-z') z'^{-1/2}, rz = 1/z', G = w sigma nu_y, D' the scaled d:
//   [g (nu.G) + g' (d.G)(d.nu)/r] = sqrt(log2 e) kappa kappa' E rz
//       [P1 (nu.G) - (ln2 P0 + 2 rz P1) (D'.G)(D'.nu) rz]
// (kappa = 1/rho, kappa' = log2(e)/rho, kappa/kappa' = ln 2); the constant
// sqrt(log2 e) kappa kappa' is applied by the caller.
struct PolyRZ2 {
    float2 c0[FIT_LONG], c1[FIT_LONG];
    __device__ __forceinline__ explicit PolyRZ2(bool short_fit) {
        const int off = short_fit ? FIT_LONG : 0;
#pragma unroll
        for (int k = 0; k < FIT_LONG; ++k) {
            const int i = min(off + k, FIT_LONG + FIT_SHORT - 1);
            const float v0 = YK_P0_F32_RZ[i], v1 = YK_P1_F32_RZ[i];
            c0[k] = make_float2(v0, v0);
            c1[k] = make_float2(v1, v1);
        }
    }
};
static_assert(sizeof(YK_P0_F32_RZ) == (FIT_LONG + FIT_SHORT) * sizeof(float), "fit lengths");

template <int NC>
__device__ __forceinline__ float2 grad2(float2 TX, float2 TY, float2 NX, float2 NY, const float4& A,
                                        const float4& B, const PolyRZ2& P, float2 acc) {
    const float2 dX = __fadd2_rn(TX, make_float2(A.x, A.y));
    const float2 dY = __fadd2_rn(TY, make_float2(A.z, A.w));
    const float2 z2 = __ffma2_rn(dX, dX, __fmul2_rn(dY, dY));
    const float2 rz = make_float2(rsqrt_fast(z2.x), rsqrt_fast(z2.y));
    const float2 zp = __fmul2_rn(z2, rz);
    float2 p0 = P.c0[NC - 1], p1 = P.c1[NC - 1];
#pragma unroll
    for (int k = NC - 2; k >= 0; --k) {
        p0 = __ffma2_rn(p0, rz, P.c0[k]);
        p1 = __ffma2_rn(p1, rz, P.c1[k]);
    }
    const float2 E = make_float2(ex2_fast(-zp.x) * rsqrt_fast(zp.x), ex2_fast(-zp.y) * rsqrt_fast(zp.y));
    const float2 Gx = make_float2(B.x, B.y), Gy = make_float2(B.z, B.w);
    const float2 nn = __ffma2_rn(NX, Gx, __fmul2_rn(NY, Gy));
    const float2 dnG = __ffma2_rn(dX, Gx, __fmul2_rn(dY, Gy));
    const float2 dnT = __ffma2_rn(dX, NX, __fmul2_rn(dY, NY));
    const float2 aneg = __ffma2_rn(make_float2(-0.69314718f, -0.69314718f), p0,
                                   __fmul2_rn(__fmul2_rn(make_float2(-2.0f, -2.0f), rz), p1));
    const float2 bneg = __fmul2_rn(__fmul2_rn(aneg, dnG), __fmul2_rn(dnT, rz));
    const float2 br = __ffma2_rn(p1, nn, bneg);
    return __ffma2_rn(__fmul2_rn(E, rz), br, acc);
}

// Pair-packed FP32 source records of one density, written once per operator
// application and read by every block of the FP32 far-field kernels: for
// source particle s and pair m (its nodes 2m, 2m + 1),
//   rec[2 (s hp + m)]     = A = (-X0, -X1, -Y0, -Y1)   (scaled offsets from
//                                                      the particle's centre)
//   rec[2 (s hp + m) + 1] = B = (g0x, g1x, g0y, g1y),  g = w sigma nu,
// hp = ceil(npp / 2); a particle with an odd node count pads its last pair
// with a far, weightless source.
__device__ __forceinline__ void src_pairs_at(const GeomView& G, const double* __restrict__ sigma,
                                             float kpf, float4* __restrict__ rec, int64_t idx) {
    const int hp = (G.npp + 1) >> 1;
    if (idx >= (int64_t)G.np * hp) return;
    const int s = (int)(idx / hp), m = (int)(idx % hp);
    float xs[2], ys[2], gx[2], gy[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = 2 * m + h;
        if (q < G.npp) {
            const int64_t j = (int64_t)s * G.npp + q;
            const float2 x = G.xi[j];
            const double ws = G.w[j] * sigma[j];
            xs[h] = -kpf * x.x;
            ys[h] = -kpf * x.y;
            gx[h] = (float)(ws * G.nx[j]);
            gy[h] = (float)(ws * G.ny[j]);
        } else {
            xs[h] = 1.0e6f;
            ys[h] = 0.0f;
            gx[h] = 0.0f;
            gy[h] = 0.0f;
        }
    }
    rec[2 * idx] = make_float4(xs[0], xs[1], ys[0], ys[1]);
    rec[2 * idx + 1] = make_float4(gx[0], gx[1], gy[0], gy[1]);
}

#ifdef YK_DEFINE_P2P_KERNELS
__global__ void k_src_pairs(GeomView G, const double* __restrict__ sigma, float kpf,
                            float4* __restrict__ rec) {
    src_pairs_at(G, sigma, kpf, rec, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}
#endif

// Stage the source pairs of nodes [jb, jb + cnt) of particle s into shared
// memory (jb even): plain 16-byte loads of the pre-packed records.
__device__ __forceinline__ void stage_rec(const float4* __restrict__ rec, int npp, int s, int jb,
                                          int cnt, float4* srcA, float4* srcB) {
    const int hp = (npp + 1) >> 1;
    const int npair = (cnt + 1) >> 1;
    const float4* r = rec + 2 * ((int64_t)s * hp + (jb >> 1));
    for (int m = threadIdx.x; m < npair; m += blockDim.x) {
        srcA[m] = r[2 * m];
        srcB[m] = r[2 * m + 1];
    }
}

// One staged tile of the normal derivative for two targets: packed far
// pairs into f0/f1 (scaled units; NC selects the fit), near/own pairs
// (scalar) into s0/s1.
template <int NC>
__device__ __forceinline__ void grad_tile(const float4* srcA, const float4* srcB, int jb, int cnt,
                                          const GeomView& G, const TargetF32& T0,
                                          const TargetF32& T1, bool use0, bool use1, float nx0,
                                          float ny0, float nx1, float ny1, float inv_kp,
                                          float kappa, float rho, const PolyRZ2& P, float& f0,
                                          float& f1, float& s0, float& s1) {
    const int npair = (cnt + 1) >> 1;
    if (use0 && use1 && !T0.close && !T1.close) {
        const float2 TX0 = make_float2(T0.TX, T0.TX), TY0 = make_float2(T0.TY, T0.TY);
        const float2 TX1 = make_float2(T1.TX, T1.TX), TY1 = make_float2(T1.TY, T1.TY);
        const float2 NX0 = make_float2(nx0, nx0), NY0 = make_float2(ny0, ny0);
        const float2 NX1 = make_float2(nx1, nx1), NY1 = make_float2(ny1, ny1);
        float2 a0 = make_float2(0.0f, 0.0f), a1 = a0;
        for (int m = 0; m < npair; ++m) {
            const float4 A = srcA[m], B = srcB[m];
            a0 = grad2<NC>(TX0, TY0, NX0, NY0, A, B, P, a0);
            a1 = grad2<NC>(TX1, TY1, NX1, NY1, A, B, P, a1);
        }
        f0 += a0.x + a0.y;
        f1 += a1.x + a1.y;
        return;
    }
    for (int q = 0; q < cnt; ++q) {
        const float4 S = src_scalar(srcA, srcB, q);
        const int pq = (jb + q) / G.ngl;
        if (use0 && !(T0.own && is_near_panel(T0.pan, pq, G.npan, G.near_w)))
            s0 += PairF32::grad((T0.TX - S.x) * inv_kp, (T0.TY - S.y) * inv_kp, nx0, ny0, S.z, S.w,
                                kappa, rho);
        if (use1 && !(T1.own && is_near_panel(T1.pan, pq, G.npan, G.near_w)))
            s1 += PairF32::grad((T1.TX - S.x) * inv_kp, (T1.TY - S.y) * inv_kp, nx1, ny1, S.z, S.w,
                                kappa, rho);
    }
}

// Packed far pairs of one staged tile for two targets (NC selects the fit).
template <int NC>
__device__ __forceinline__ void far_tile(const float4* srcA, const float4* srcB, int npair,
                                         const TargetF32& T0, const TargetF32& T1,
                                         const PolyRZ& P, float& r0, float& r1) {
    const float2 TX0 = make_float2(T0.TX, T0.TX), TY0 = make_float2(T0.TY, T0.TY);
    const float2 TX1 = make_float2(T1.TX, T1.TX), TY1 = make_float2(T1.TY, T1.TY);
    float2 a0 = make_float2(0.0f, 0.0f), a1 = a0;
#pragma unroll 2
    for (int m = 0; m < npair; ++m) {
        const float4 A = srcA[m], B = srcB[m];
        a0 = far2<NC>(TX0, TY0, A, B, P, a0);
        a1 = far2<NC>(TX1, TY1, A, B, P, a1);
    }
    r0 = a0.x + a0.y;
    r1 = a1.x + a1.y;
}

#ifdef YK_DEFINE_P2P_KERNELS
template <bool MASK>
__global__ void __launch_bounds__(F32_TPB, 8) k_p2p_f32(GeomView G, const float4* __restrict__ rec,
                                                     int ppc, float kscale, double skip_gap,
                                                     bool own_by_block,
                                                     double* __restrict__ partial) {
    __shared__ float4 srcA[STILE / 2], srcB[STILE / 2];
    const int64_t i0 = blockIdx.x * (int64_t)TPB + threadIdx.x;
    const int64_t i1 = i0 + F32_TPB;
    const bool act0 = i0 < G.n, act1 = i1 < G.n;
    const int64_t ii0 = act0 ? i0 : 0, ii1 = act1 ? i1 : 0;
    const float2 xi0 = G.xi[ii0], xi1 = G.xi[ii1];
    const int pt0 = (int)(ii0 / G.npp), pt1 = (int)(ii1 / G.npp);
    const int pan0 = (int)(ii0 % G.npp) / G.ngl, pan1 = (int)(ii1 % G.npp) / G.ngl;
    const float kpf = (float)(LOG2E / G.rho);          // log2(e) / rho
    const float near_gap = 2.0f * (float)G.rho * 1.0001f + 1e-4f;  // z <= 2 possible below
    const float short_gap = Z_SHORT * (float)G.rho, zero_gap = ZP_ZERO / kpf;
    const int pa = (int)(blockIdx.x * (int64_t)TPB / G.npp);
    const int pb = (int)((min((int64_t)G.n, (blockIdx.x + 1) * (int64_t)TPB) - 1) / G.npp);
    const int s0 = blockIdx.y * ppc;
    const int s1 = min(G.np, s0 + ppc);
    double acc0 = 0.0, acc1 = 0.0;
    for (int s = s0; s < s1; ++s) {
        const PairRange rg = block_range(G, pa, pb, s);
        if (rg.gap >= zero_gap) continue;   // every pair adds +0 in FP32 (block-uniform)
        float rc;
        const int mode = far_mode(rg, short_gap, kpf, rc);
        const PolyRZ P(mode, rc);
        TargetF32 T0, T1;
        target_setup(T0, G, pt0, s, xi0, kpf, near_gap, MASK, skip_gap, pan0);
        target_setup(T1, G, pt1, s, xi1, kpf, near_gap, MASK, skip_gap, pan1);
        // a target skips the source particle when the FP64 tiles hold the pair
        // (MASK) or when it is the target's own particle and the self block
        // adds it (own_by_block); the particle is skipped only when every
        // thread of the block agrees (a block-wide vote reached by all
        // threads), so barriers stay uniform
        const bool skip0 = (MASK && T0.skip) || (own_by_block && T0.own);
        const bool skip1 = (MASK && T1.skip) || (own_by_block && T1.own);
        const bool block_skip = (MASK || own_by_block) ? __syncthreads_and(skip0 && skip1) : false;
        if (block_skip) continue;
        for (int jb = 0; jb < G.npp; jb += STILE) {
            const int cnt = min(STILE, G.npp - jb);
            const int npair = (cnt + 1) >> 1;
            __syncthreads();
            stage_rec(rec, G.npp, s, jb, cnt, srcA, srcB);
            __syncthreads();
            float r0 = 0.0f, r1 = 0.0f;
            if (!T0.close && !T1.close && !skip0 && !skip1) {
                if (mode == NARROW3) far_tile<NARROW3>(srcA, srcB, npair, T0, T1, P, r0, r1);
                else if (mode == NARROW) far_tile<NARROW>(srcA, srcB, npair, T0, T1, P, r0, r1);
                else if (mode == FIT_SHORT) far_tile<FIT_SHORT>(srcA, srcB, npair, T0, T1, P, r0, r1);
                else far_tile<FIT_LONG>(srcA, srcB, npair, T0, T1, P, r0, r1);
            } else {
                for (int q = 0; q < cnt; ++q) {
                    const float4 S = src_scalar(srcA, srcB, q);
                    const int pq = (jb + q) / G.ngl;
                    if (!skip0 && !(T0.own && is_near_panel(T0.pan, pq, G.npan, G.near_w)))
                        r0 += PairF32::any(T0.TX - S.x, T0.TY - S.y, S.z, S.w);
                    if (!skip1 && !(T1.own && is_near_panel(T1.pan, pq, G.npan, G.near_w)))
                        r1 += PairF32::any(T1.TX - S.x, T1.TY - S.y, S.z, S.w);
                }
            }
            acc0 += (double)r0;
            acc1 += (double)r1;
        }
    }
    if (act0) partial[blockIdx.y * G.n + i0] = acc0 * (double)kscale;
    if (act1) partial[blockIdx.y * G.n + i1] = acc1 * (double)kscale;
}
#endif

// ---------------------------------------------------------------------------
// Symmetric FP32 far field of the dense operator (k_p2p_f32_sym).
//
// For nodes i of particle P and j of particle Q, d = x_i - y_j and
// g = w sigma nu, the two double-layer terms (Eq. double-layer-def) are
//   K(x_i, y_j) g_j = c(r) (d . g_j),   K(y_j, x_i) g_i = c(r) (-d . g_i),
// with the same radial factor c(r) = K1(r/rho) / (2 pi rho r), which carries
// all the special-function work (1/z', exp2, the K1 fit or expansion). The
// kernel takes a list of particle pairs (P, Q), P < Q, sorted by P, and
// evaluates c once per node pair for both directions: about 10 FMA-pipe lane
// operations and 1.5 MUFU operations per interaction instead of 17 and 3.
//
// Per block: 128 threads, SYM_TASKS consecutive pairs of the list. P's nodes
// sit in registers (warp w holds nodes 64 w + l and 64 w + 32 + l of the
// chunk in lane l), Q's nodes in shared memory as the packed source records
// (two nodes per record). Q's side rotates: in group b of 32 records, at
// step k lane l evaluates record 32 b + ((l + k) mod 32), so the 32 lanes
// read 32 distinct records (no bank conflicts) and each record's reverse
// sums are held by exactly one lane. After every step each lane passes its
// reverse sums to lane l - 1 (a warp shuffle); after 32 steps every record's
// sums are back in lane (record mod 32), complete over the warp's 64 nodes
// of P. The four warps' sums are added in shared memory and go to Q's nodes;
// P's sums stay in FP64 registers while consecutive pairs share P. Both go
// to an FP64 buffer by atomic adds (the order of those adds, and so the last
// bits of the result, vary from run to run).
//
// Particle-pair classes as in k_p2p_f32 (same FP32 arithmetic on the pair's
// range [gap, far]): pairs whose every term is an exact FP32 zero are not
// listed; close pairs (gap <= 2 rho) evaluate pairs with z <= 2 by the K1
// series; otherwise the full or short fit or the narrow expansions.
// ---------------------------------------------------------------------------
constexpr int SYM_TASKS = 8;     // particle pairs per block
constexpr int CLOSE = 8;         // pair mode: some node pairs may have z <= 2

// The radial factor of two packed pairs (one target, two sources) in the
// units of PairF32::far without the dot product, and the scaled separations.
template <int NC>
__device__ __forceinline__ float2 coef2(float2 TX, float2 TY, const float4& A, const PolyRZ& P,
                                        float2& dX, float2& dY) {
    dX = __fadd2_rn(TX, make_float2(A.x, A.y));
    dY = __fadd2_rn(TY, make_float2(A.z, A.w));
    const float2 z2 = __ffma2_rn(dX, dX, __fmul2_rn(dY, dY));
    const float2 rz = make_float2(rsqrt_fast(z2.x), rsqrt_fast(z2.y));   // 1/z'
    const float2 zp = __fmul2_rn(z2, rz);                                 // z'
    if constexpr (NC == NARROW || NC == NARROW3) {
        const float2 u = __ffma2_rn(rz, P.c[5], P.c[6]);                  // rz/rc - 1
        constexpr int top = (NC == NARROW) ? 4 : 3;
        float2 q = P.c[top];
#pragma unroll
        for (int k = top - 1; k >= 0; --k) q = __ffma2_rn(q, u, P.c[k]); // rz^{1/2} P1(rz)
        const float2 e = make_float2(ex2_fast(-zp.x), ex2_fast(-zp.y));
        return __fmul2_rn(__fmul2_rn(e, q), rz);
    } else {
        float2 p = P.c[NC - 1];
#pragma unroll
        for (int k = NC - 2; k >= 0; --k) p = __ffma2_rn(p, rz, P.c[k]); // P1 in rz
        const float2 e = make_float2(ex2_fast(-zp.x), ex2_fast(-zp.y));
        const float2 sq = make_float2(rsqrt_fast(zp.x), rsqrt_fast(zp.y));   // z'^{-1/2}
        return __fmul2_rn(__fmul2_rn(__fmul2_rn(e, p), sq), rz);
    }
}

// The radial factor of one pair for any z (the series of PairF32::any for
// z <= 2), same units as coef2.
__device__ __forceinline__ float coef_any(float dX, float dY) {
    const float z2 = fmaf(dX, dX, dY * dY);
    const float rz = rsqrt_fast(z2);
    const float zp = z2 * rz;
    const float z = zp * (1.0f / LOG2E_F);
    if (z > 2.0f) {
        const float s = fmaf(4.0f * LOG2E_F, rz, -1.0f);     // 2t - 1
        const float P = hornerf(YK_P1_F32, s);
        return (ex2_fast(-zp) * P * rsqrt_fast(zp)) * rz;
    }
    return k1f(z, 2.0f / z) * rsqrtf(LOG2E_F) * rz;
}

// One target against one packed record (two sources): forward sums into fw
// (one lane per source), reverse sums of the two sources into rv. NG = -g of
// the target, in both lanes.
template <int NC>
__device__ __forceinline__ void sym_pair(float2 TX, float2 TY, float2 NGX, float2 NGY,
                                         const float4& A, const float4& B, const PolyRZ& P,
                                         float2& fw, float2& rv) {
    float2 dX, dY, c;
    if constexpr (NC == CLOSE) {
        dX = __fadd2_rn(TX, make_float2(A.x, A.y));
        dY = __fadd2_rn(TY, make_float2(A.z, A.w));
        const float z2x = fmaf(dX.x, dX.x, dY.x * dY.x), z2y = fmaf(dX.y, dX.y, dY.y * dY.y);
        if (z2x > ZCUT2 && z2y > ZCUT2) c = coef2<FIT_LONG>(TX, TY, A, P, dX, dY);
        else c = make_float2(coef_any(dX.x, dY.x), coef_any(dX.y, dY.y));
    } else {
        c = coef2<NC>(TX, TY, A, P, dX, dY);
    }
    const float2 dj = __ffma2_rn(dX, make_float2(B.x, B.y), __fmul2_rn(dY, make_float2(B.z, B.w)));
    const float2 di = __ffma2_rn(dX, NGX, __fmul2_rn(dY, NGY));
    fw = __ffma2_rn(c, dj, fw);
    rv = __ffma2_rn(c, di, rv);
}

// All rotation groups of one staged chunk of Q for the lane's two targets.
template <int NC>
__device__ __forceinline__ void sym_chunk(const float4* qA, const float4* qB, int ngrp, int lane,
                                          float TX0, float TY0, float TX1, float TY1, float NGX0,
                                          float NGY0, float NGX1, float NGY1, const PolyRZ& P,
                                          float2& fw0, float2& fw1, float* rsum_w) {
    const float2 tx0 = make_float2(TX0, TX0), ty0 = make_float2(TY0, TY0);
    const float2 tx1 = make_float2(TX1, TX1), ty1 = make_float2(TY1, TY1);
    const float2 ngx0 = make_float2(NGX0, NGX0), ngy0 = make_float2(NGY0, NGY0);
    const float2 ngx1 = make_float2(NGX1, NGX1), ngy1 = make_float2(NGY1, NGY1);
    const int next = (lane + 1) & 31;
    for (int b = 0; b < ngrp; ++b) {
        float2 rv = make_float2(0.0f, 0.0f);
#pragma unroll 2
        for (int k = 0; k < 32; ++k) {
            const int m = 32 * b + ((lane + k) & 31);
            const float4 A = qA[m], B = qB[m];
            sym_pair<NC>(tx0, ty0, ngx0, ngy0, A, B, P, fw0, rv);
            sym_pair<NC>(tx1, ty1, ngx1, ngy1, A, B, P, fw1, rv);
            rv.x = __shfl_sync(0xffffffffu, rv.x, next);
            rv.y = __shfl_sync(0xffffffffu, rv.y, next);
        }
        // record 32 b + lane: Q nodes 64 b + 2 lane and 64 b + 2 lane + 1 of the chunk
        rsum_w[64 * b + 2 * lane] = rv.x;
        rsum_w[64 * b + 2 * lane + 1] = rv.y;
    }
}

// Work item w: pair w / (npc nqc), chunk (w / nqc) mod npc of 256 of P's
// nodes, and range w mod nqc of qch of Q's nodes (qch a multiple of 64, at
// most 256; smaller ranges give small systems enough blocks). A block takes
// ipb consecutive items.
template <bool ALL>   // ALL: every warp of the block holds targets (nw = F32_TPB / 32)
__device__ __forceinline__ void sym_items(const GeomView& G, const float4* __restrict__ rec,
                                          const int2* __restrict__ tasks, int ntasks, int qch,
                                          int ipb, int nw, double kscale,
                                          double* __restrict__ out, int block) {
    __shared__ float4 qA[STILE / 2], qB[STILE / 2];
    __shared__ float rsum[F32_TPB / 32][STILE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool wact = ALL || warp < nw;   // nw warps hold a chunk of 64 nw of P's nodes
    const float kpf = (float)(LOG2E / G.rho);
    const float near_gap = 2.0f * (float)G.rho * 1.0001f + 1e-4f;
    const float short_gap = Z_SHORT * (float)G.rho;
    const int hp = (G.npp + 1) >> 1;
    const int csz = ALL ? STILE : 64 * nw;
    const int npc = (G.npp + csz - 1) / csz, nqc = (G.npp + qch - 1) / qch;
    const int64_t items = (int64_t)ntasks * npc * nqc;
    const int64_t w0 = (int64_t)block * ipb, w1 = min(items, w0 + ipb);
    const int lt0 = 64 * warp + lane, lt1 = lt0 + 32;   // the lane's targets in a chunk
    int curP = -1, curC = 0;                            // owner of the FP64 forward sums
    double f0 = 0.0, f1 = 0.0;
    for (int64_t w = w0; w < w1; ++w) {
        const int t = (int)(w / ((int64_t)npc * nqc));
        const int pc = (int)((w / nqc) % npc) * csz;
        const int qc = (int)(w % nqc) * qch;
        const int2 pq = tasks[t];
        const int P = pq.x, Q = pq.y;
        const PairRange rg = block_range(G, P, P, Q);   // block-uniform
        float rc = 0.0f;
        const int mode = (rg.gap <= near_gap) ? CLOSE : far_mode(rg, short_gap, kpf, rc);
        const PolyRZ Pz(mode == CLOSE ? FIT_LONG : mode, rc);
        const float4 cp = G.c32[P], cq = G.c32[Q];
        const float oX = kpf * ((cp.x - cq.x) + (cp.z - cq.z));
        const float oY = kpf * ((cp.y - cq.y) + (cp.w - cq.w));
        {
            if (P != curP || pc != curC) {
                if (curP >= 0) {
                    const int64_t b = (int64_t)curP * G.npp + curC;
                    if (wact && curC + lt0 < G.npp) atomicAdd(&out[b + lt0], f0 * kscale);
                    if (wact && curC + lt1 < G.npp) atomicAdd(&out[b + lt1], f1 * kscale);
                }
                curP = P;
                curC = pc;
                f0 = f1 = 0.0;
            }
            // the lane's two targets of P: scaled position relative to Q's centre, -g
            float TX[2], TY[2], NGX[2], NGY[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int li = pc + (h ? lt1 : lt0);
                if (wact && li < G.npp) {
                    const int64_t r = 2 * ((int64_t)P * hp + (li >> 1));
                    const float4 A = rec[r], B = rec[r + 1];
                    const bool odd = li & 1;
                    TX[h] = oX - (odd ? A.y : A.x);
                    TY[h] = oY - (odd ? A.w : A.z);
                    NGX[h] = -(odd ? B.y : B.x);
                    NGY[h] = -(odd ? B.w : B.z);
                } else {   // no node: far away and weightless
                    TX[h] = 3.0e6f;
                    TY[h] = 0.0f;
                    NGX[h] = NGY[h] = 0.0f;
                }
            }
            {
                const int cnt = min(qch, G.npp - qc);
                const int npair = (cnt + 1) >> 1;
                const int ngrp = (npair + 31) >> 5;
                __syncthreads();   // previous chunk's shared data fully used
                const float4* rq = rec + 2 * ((int64_t)Q * hp + (qc >> 1));
                for (int m = threadIdx.x; m < 32 * ngrp; m += blockDim.x) {
                    if (m < npair) {
                        qA[m] = rq[2 * m];
                        qB[m] = rq[2 * m + 1];
                    } else {       // padding records: far away and weightless
                        qA[m] = make_float4(1.0e6f, 1.0e6f, 0.0f, 0.0f);
                        qB[m] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    }
                }
                __syncthreads();
                float2 fw0 = make_float2(0.0f, 0.0f), fw1 = fw0;
                float* rw = rsum[warp];
                if (wact) switch (mode) {
                    case NARROW3:
                        sym_chunk<NARROW3>(qA, qB, ngrp, lane, TX[0], TY[0], TX[1], TY[1], NGX[0],
                                           NGY[0], NGX[1], NGY[1], Pz, fw0, fw1, rw);
                        break;
                    case NARROW:
                        sym_chunk<NARROW>(qA, qB, ngrp, lane, TX[0], TY[0], TX[1], TY[1], NGX[0],
                                          NGY[0], NGX[1], NGY[1], Pz, fw0, fw1, rw);
                        break;
                    case FIT_SHORT:
                        sym_chunk<FIT_SHORT>(qA, qB, ngrp, lane, TX[0], TY[0], TX[1], TY[1],
                                             NGX[0], NGY[0], NGX[1], NGY[1], Pz, fw0, fw1, rw);
                        break;
                    case CLOSE:
                        sym_chunk<CLOSE>(qA, qB, ngrp, lane, TX[0], TY[0], TX[1], TY[1], NGX[0],
                                         NGY[0], NGX[1], NGY[1], Pz, fw0, fw1, rw);
                        break;
                    default:
                        sym_chunk<FIT_LONG>(qA, qB, ngrp, lane, TX[0], TY[0], TX[1], TY[1],
                                            NGX[0], NGY[0], NGX[1], NGY[1], Pz, fw0, fw1, rw);
                }
                f0 += (double)(fw0.x + fw0.y);
                f1 += (double)(fw1.x + fw1.y);
                __syncthreads();   // every warp's reverse sums are in rsum
                for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
                    float v;
                    if (ALL) {
                        v = (rsum[0][j] + rsum[1][j]) + (rsum[2][j] + rsum[3][j]);
                    } else {
                        v = rsum[0][j];
                        for (int q = 1; q < nw; ++q) v += rsum[q][j];
                    }
                    atomicAdd(&out[(int64_t)Q * G.npp + qc + j], (double)v * kscale);
                }
            }
        }
    }
    if (curP >= 0) {
        const int64_t b = (int64_t)curP * G.npp + curC;
        if (wact && curC + lt0 < G.npp) atomicAdd(&out[b + lt0], f0 * kscale);
        if (wact && curC + lt1 < G.npp) atomicAdd(&out[b + lt1], f1 * kscale);
    }
}

#ifdef YK_DEFINE_P2P_KERNELS
// ALL: blocks of F32_TPB threads, every warp with targets; otherwise nw
// warps (particles of at most 64 nw nodes)
template <bool ALL>
__global__ void __launch_bounds__(F32_TPB, 6) k_p2p_f32_sym(GeomView G, const float4* __restrict__ rec,
                                                           const int2* __restrict__ tasks,
                                                           int ntasks, int qch, int ipb, int nw,
                                                           double kscale,
                                                           double* __restrict__ out) {
    sym_items<ALL>(G, rec, tasks, ntasks, qch, ipb, nw, kscale, out, blockIdx.x);
}
#endif

// ---------------------------------------------------------------------------
// Symmetric FP32 far field of the normal derivative (k_p2p_f32_symg).
//
// For nodes i of P and j of Q, d = x_i - y_j, the normal-derivative kernel
//   H(i, j) = g(r) (nu_i . nu_j) + g'(r) (d . nu_j)(d . nu_i) / r,
//   g = K1(r/rho) / (rho r) (2 pi left out),
// is symmetric: the term of node j at node i is H q_j and that of node i at
// node j is H q_i (q = w sigma). One evaluation of H serves both directions.
// The records carry the normals and q separately: per pair of nodes A =
// scaled offsets (as for the value kernel), B = (nu0x, nu1x, nu0y, nu1y),
// C = (q0, q1, 0, 0). The work items, the staging of Q, the rotation of the
// reverse sums and the FP64 atomic outputs are those of k_p2p_f32_sym; the
// fits are those of k_p2p_f32_grad (long or short in rz); close pairs
// (z <= 2 possible) evaluate such node pairs by PairF32::grad.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void src_grad_pairs_at(const GeomView& G,
                                                  const double* __restrict__ sigma, float kpf,
                                                  float4* __restrict__ rec, int64_t idx) {
    const int hp = (G.npp + 1) >> 1;
    if (idx >= (int64_t)G.np * hp) return;
    const int s = (int)(idx / hp), m = (int)(idx % hp);
    float xs[2], ys[2], nx[2], ny[2], q[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = 2 * m + h;
        if (k < G.npp) {
            const int64_t j = (int64_t)s * G.npp + k;
            const float2 x = G.xi[j];
            xs[h] = -kpf * x.x;
            ys[h] = -kpf * x.y;
            nx[h] = (float)G.nx[j];
            ny[h] = (float)G.ny[j];
            q[h] = (float)(G.w[j] * sigma[j]);
        } else {
            xs[h] = 1.0e6f;
            ys[h] = 0.0f;
            nx[h] = ny[h] = q[h] = 0.0f;
        }
    }
    rec[3 * idx] = make_float4(xs[0], xs[1], ys[0], ys[1]);
    rec[3 * idx + 1] = make_float4(nx[0], nx[1], ny[0], ny[1]);
    rec[3 * idx + 2] = make_float4(q[0], q[1], 0.0f, 0.0f);
}

#ifdef YK_DEFINE_P2P_KERNELS
__global__ void k_src_grad_pairs(GeomView G, const double* __restrict__ sigma, float kpf,
                                 float4* __restrict__ rec) {
    src_grad_pairs_at(G, sigma, kpf, rec, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}
#endif

// Constants of the symmetric normal derivative: the scaled units of the fit
// path times cf = sqrt(log2 e) kappa kappa' are physical (2 pi left out).
struct SymGradC {
    float inv_kp, kappa, rho, icf;   // 1/kappa', 1/rho, rho, 1/cf
};

// H of one node pair in the fit path's units, any z: the long fit for
// z > 2, else PairF32::grad (physical units) times 1/cf.
__device__ __forceinline__ float hsym_any(float dX, float dY, float ntx, float nty, float nsx,
                                          float nsy, const SymGradC& K) {
    const float z2 = fmaf(dX, dX, dY * dY);
    if (z2 > ZCUT2) {
        const float rz = rsqrt_fast(z2);
        const float zp = z2 * rz;
        float p0 = YK_P0_F32_RZ[FIT_LONG - 1], p1 = YK_P1_F32_RZ[FIT_LONG - 1];
#pragma unroll
        for (int k = FIT_LONG - 2; k >= 0; --k) {
            p0 = fmaf(p0, rz, YK_P0_F32_RZ[k]);
            p1 = fmaf(p1, rz, YK_P1_F32_RZ[k]);
        }
        const float E = ex2_fast(-zp) * rsqrt_fast(zp);
        const float nn = fmaf(ntx, nsx, nty * nsy);
        const float ds = fmaf(dX, nsx, dY * nsy), dt = fmaf(dX, ntx, dY * nty);
        const float a = fmaf(-0.69314718f, p0, -2.0f * rz * p1);
        return E * rz * fmaf(p1, nn, a * ds * dt * rz);
    }
    return PairF32::grad(dX * K.inv_kp, dY * K.inv_kp, ntx, nty, nsx, nsy, K.kappa, K.rho) * K.icf;
}

template <int NC>
__device__ __forceinline__ void symg_pair(float2 TX, float2 TY, float2 NX, float2 NY, float2 QT,
                                          const float4& A, const float4& B, const float4& C,
                                          const PolyRZ2& P, const SymGradC& K, float2& fw,
                                          float2& rv) {
    const float2 dX = __fadd2_rn(TX, make_float2(A.x, A.y));
    const float2 dY = __fadd2_rn(TY, make_float2(A.z, A.w));
    const float2 Bx = make_float2(B.x, B.y), By = make_float2(B.z, B.w);
    float2 H;
    if constexpr (NC == CLOSE) {
        H.x = hsym_any(dX.x, dY.x, NX.x, NY.x, B.x, B.z, K);
        H.y = hsym_any(dX.y, dY.y, NX.y, NY.y, B.y, B.w, K);
    } else {
        const float2 z2 = __ffma2_rn(dX, dX, __fmul2_rn(dY, dY));
        const float2 rz = make_float2(rsqrt_fast(z2.x), rsqrt_fast(z2.y));
        const float2 zp = __fmul2_rn(z2, rz);
        float2 p0 = P.c0[NC - 1], p1 = P.c1[NC - 1];
#pragma unroll
        for (int k = NC - 2; k >= 0; --k) {
            p0 = __ffma2_rn(p0, rz, P.c0[k]);
            p1 = __ffma2_rn(p1, rz, P.c1[k]);
        }
        const float2 E = make_float2(ex2_fast(-zp.x) * rsqrt_fast(zp.x),
                                     ex2_fast(-zp.y) * rsqrt_fast(zp.y));
        const float2 nn = __ffma2_rn(NX, Bx, __fmul2_rn(NY, By));
        const float2 ds = __ffma2_rn(dX, Bx, __fmul2_rn(dY, By));
        const float2 dt = __ffma2_rn(dX, NX, __fmul2_rn(dY, NY));
        const float2 a = __ffma2_rn(make_float2(-0.69314718f, -0.69314718f), p0,
                                    __fmul2_rn(__fmul2_rn(make_float2(-2.0f, -2.0f), rz), p1));
        const float2 br = __ffma2_rn(p1, nn, __fmul2_rn(__fmul2_rn(a, ds), __fmul2_rn(dt, rz)));
        H = __fmul2_rn(__fmul2_rn(E, rz), br);
    }
    fw = __ffma2_rn(H, make_float2(C.x, C.y), fw);
    rv = __ffma2_rn(H, QT, rv);
}

template <int NC>
__device__ __forceinline__ void symg_chunk(const float4* qA, const float4* qB, const float4* qC,
                                           int ngrp, int lane, const float* TX, const float* TY,
                                           const float* NX, const float* NY, const float* QT,
                                           const PolyRZ2& P, const SymGradC& K, float2& fw0,
                                           float2& fw1, float* rsum_w) {
    const float2 tx0 = make_float2(TX[0], TX[0]), ty0 = make_float2(TY[0], TY[0]);
    const float2 tx1 = make_float2(TX[1], TX[1]), ty1 = make_float2(TY[1], TY[1]);
    const float2 nx0 = make_float2(NX[0], NX[0]), ny0 = make_float2(NY[0], NY[0]);
    const float2 nx1 = make_float2(NX[1], NX[1]), ny1 = make_float2(NY[1], NY[1]);
    const float2 q0 = make_float2(QT[0], QT[0]), q1 = make_float2(QT[1], QT[1]);
    const int next = (lane + 1) & 31;
    for (int b = 0; b < ngrp; ++b) {
        float2 rv = make_float2(0.0f, 0.0f);
#pragma unroll 2
        for (int k = 0; k < 32; ++k) {
            const int m = 32 * b + ((lane + k) & 31);
            const float4 A = qA[m], B = qB[m], C = qC[m];
            symg_pair<NC>(tx0, ty0, nx0, ny0, q0, A, B, C, P, K, fw0, rv);
            symg_pair<NC>(tx1, ty1, nx1, ny1, q1, A, B, C, P, K, fw1, rv);
            rv.x = __shfl_sync(0xffffffffu, rv.x, next);
            rv.y = __shfl_sync(0xffffffffu, rv.y, next);
        }
        rsum_w[64 * b + 2 * lane] = rv.x;
        rsum_w[64 * b + 2 * lane + 1] = rv.y;
    }
}

#ifdef YK_DEFINE_P2P_KERNELS
template <bool ALL>   // as k_p2p_f32_sym
__global__ void __launch_bounds__(F32_TPB, 5) k_p2p_f32_symg(GeomView G,
                                                            const float4* __restrict__ rec,
                                                            const int2* __restrict__ tasks,
                                                            int ntasks, int qch, int ipb, int nw,
                                                            double kscale,
                                                            double* __restrict__ out) {
    __shared__ float4 qA[STILE / 2], qB[STILE / 2], qC[STILE / 2];
    __shared__ float rsum[F32_TPB / 32][STILE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool wact = ALL || warp < nw;   // nw warps hold a chunk of 64 nw of P's nodes
    const float kpf = (float)(LOG2E / G.rho);
    const float near_gap = 2.0f * (float)G.rho * 1.0001f + 1e-4f;
    const float short_gap = Z_SHORT * (float)G.rho;
    SymGradC K;
    K.inv_kp = (float)(G.rho / LOG2E);
    K.kappa = (float)(1.0 / G.rho);
    K.rho = (float)G.rho;
    K.icf = (float)(1.0 / (sqrt(LOG2E) * (1.0 / G.rho) * (LOG2E / G.rho)));
    const int hp = (G.npp + 1) >> 1;
    const int csz = ALL ? STILE : 64 * nw;
    const int npc = (G.npp + csz - 1) / csz, nqc = (G.npp + qch - 1) / qch;
    const int64_t items = (int64_t)ntasks * npc * nqc;
    const int64_t w0 = (int64_t)blockIdx.x * ipb, w1 = min(items, w0 + ipb);
    const int lt0 = 64 * warp + lane, lt1 = lt0 + 32;
    int curP = -1, curC = 0;
    double f0 = 0.0, f1 = 0.0;
    for (int64_t w = w0; w < w1; ++w) {
        const int t = (int)(w / ((int64_t)npc * nqc));
        const int pc = (int)((w / nqc) % npc) * csz;
        const int qc = (int)(w % nqc) * qch;
        const int2 pq = tasks[t];
        const int P = pq.x, Q = pq.y;
        const PairRange rg = block_range(G, P, P, Q);   // block-uniform
        const int mode = (rg.gap <= near_gap) ? CLOSE : (rg.gap >= short_gap ? FIT_SHORT : FIT_LONG);
        const PolyRZ2 Pz(mode == FIT_SHORT);
        const float4 cp = G.c32[P], cq = G.c32[Q];
        const float oX = kpf * ((cp.x - cq.x) + (cp.z - cq.z));
        const float oY = kpf * ((cp.y - cq.y) + (cp.w - cq.w));
        if (P != curP || pc != curC) {
            if (curP >= 0) {
                const int64_t b = (int64_t)curP * G.npp + curC;
                if (wact && curC + lt0 < G.npp) atomicAdd(&out[b + lt0], f0 * kscale);
                if (wact && curC + lt1 < G.npp) atomicAdd(&out[b + lt1], f1 * kscale);
            }
            curP = P;
            curC = pc;
            f0 = f1 = 0.0;
        }
        float TX[2], TY[2], NX[2], NY[2], QT[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int li = pc + (h ? lt1 : lt0);
            if (wact && li < G.npp) {
                const int64_t r = 3 * ((int64_t)P * hp + (li >> 1));
                const float4 A = rec[r], B = rec[r + 1], C = rec[r + 2];
                const bool odd = li & 1;
                TX[h] = oX - (odd ? A.y : A.x);
                TY[h] = oY - (odd ? A.w : A.z);
                NX[h] = odd ? B.y : B.x;
                NY[h] = odd ? B.w : B.z;
                QT[h] = odd ? C.y : C.x;
            } else {   // no node: far away and weightless
                TX[h] = 3.0e6f;
                TY[h] = 0.0f;
                NX[h] = NY[h] = QT[h] = 0.0f;
            }
        }
        const int cnt = min(qch, G.npp - qc);
        const int npair = (cnt + 1) >> 1;
        const int ngrp = (npair + 31) >> 5;
        __syncthreads();   // previous chunk's shared data fully used
        const float4* rq = rec + 3 * ((int64_t)Q * hp + (qc >> 1));
        for (int m = threadIdx.x; m < 32 * ngrp; m += blockDim.x) {
            if (m < npair) {
                qA[m] = rq[3 * m];
                qB[m] = rq[3 * m + 1];
                qC[m] = rq[3 * m + 2];
            } else {       // padding records: far away and weightless
                qA[m] = make_float4(1.0e6f, 1.0e6f, 0.0f, 0.0f);
                qB[m] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                qC[m] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        }
        __syncthreads();
        float2 fw0 = make_float2(0.0f, 0.0f), fw1 = fw0;
        float* rw = rsum[warp];
        if (!wact) {
        } else if (mode == CLOSE)
            symg_chunk<CLOSE>(qA, qB, qC, ngrp, lane, TX, TY, NX, NY, QT, Pz, K, fw0, fw1, rw);
        else if (mode == FIT_SHORT)
            symg_chunk<FIT_SHORT>(qA, qB, qC, ngrp, lane, TX, TY, NX, NY, QT, Pz, K, fw0, fw1, rw);
        else
            symg_chunk<FIT_LONG>(qA, qB, qC, ngrp, lane, TX, TY, NX, NY, QT, Pz, K, fw0, fw1, rw);
        f0 += (double)(fw0.x + fw0.y);
        f1 += (double)(fw1.x + fw1.y);
        __syncthreads();   // every warp's reverse sums are in rsum
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
            float v;
            if (ALL) {
                v = (rsum[0][j] + rsum[1][j]) + (rsum[2][j] + rsum[3][j]);
            } else {
                v = rsum[0][j];
                for (int q = 1; q < nw; ++q) v += rsum[q][j];
            }
            atomicAdd(&out[(int64_t)Q * G.npp + qc + j], (double)v * kscale);
        }
    }
    if (curP >= 0) {
        const int64_t b = (int64_t)curP * G.npp + curC;
        if (wact && curC + lt0 < G.npp) atomicAdd(&out[b + lt0], f0 * kscale);
        if (wact && curC + lt1 < G.npp) atomicAdd(&out[b + lt1], f1 * kscale);
    }
}
#endif

// Particle pairs of the symmetric far field: P < Q, not every term an exact
// FP32 zero (the kernels' FP32 gap test), and, with a skip distance, not a
// pair of the FP64 tiles. Counted per P, then listed in order of Q.
__device__ __forceinline__ bool sym_pair_listed(const GeomView& G, int P, int Q, float zero_gap,
                                                bool mask, double skip_gap) {
    if (block_range(G, P, P, Q).gap >= zero_gap) return false;
    return !(mask && pair_in_tiles(G.part[P], G.part[Q], skip_gap));
}

// One warp per particle P (lanes over Q, 32 at a time); the fill writes each
// P's pairs in order of Q from the ballot of the lanes.
#ifdef YK_DEFINE_P2P_KERNELS
__global__ void k_sym_count(GeomView G, bool mask, double skip_gap, int* __restrict__ counts) {
    const int P = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (P >= G.np) return;   // warp-uniform
    const float zero_gap = ZP_ZERO / (float)(LOG2E / G.rho);
    int c = 0;
    for (int Q0 = P + 1; Q0 < G.np; Q0 += 32) {
        const int Q = Q0 + lane;
        const bool hit = Q < G.np && sym_pair_listed(G, P, Q, zero_gap, mask, skip_gap);
        c += __popc(__ballot_sync(0xffffffffu, hit));
    }
    if (lane == 0) counts[P] = c;
}
#endif

#ifdef YK_DEFINE_P2P_KERNELS
__global__ void k_sym_fill(GeomView G, bool mask, double skip_gap, const int* __restrict__ off,
                           int2* __restrict__ tasks) {
    const int P = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (P >= G.np) return;   // warp-uniform
    const float zero_gap = ZP_ZERO / (float)(LOG2E / G.rho);
    int k = off[P];
    for (int Q0 = P + 1; Q0 < G.np; Q0 += 32) {
        const int Q = Q0 + lane;
        const bool hit = Q < G.np && sym_pair_listed(G, P, Q, zero_gap, mask, skip_gap);
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) tasks[k + __popc(m & ((1u << lane) - 1u))] = make_int2(P, Q);
        k += __popc(m);
    }
}
#endif

// Pairs of the symmetric kernel from per-particle neighbour lists (the FMM
// near lists, the cut-off neighbour lists): Q in near(P), Q > P, not every
// term an exact FP32 zero, and with a skip distance not a pair of the FP64
// tiles; one warp per P, in the order of P's list.
#ifdef YK_DEFINE_P2P_KERNELS
template <bool FILL>
__global__ void k_sym_near(GeomView G, const int* __restrict__ near_off,
                           const int* __restrict__ near, bool mask, double skip_gap,
                           int* __restrict__ counts, const int* __restrict__ off,
                           int2* __restrict__ tasks) {
    const int P = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (P >= G.np) return;   // warp-uniform
    const float zero_gap = ZP_ZERO / (float)(LOG2E / G.rho);
    const int e0 = near_off[P], e1 = near_off[P + 1];
    int k = FILL ? off[P] : 0;
    for (int b = e0; b < e1; b += 32) {
        const int e = b + lane;
        const int Q = e < e1 ? near[e] : -1;
        const bool hit = Q > P && sym_pair_listed(G, P, Q, zero_gap, mask, skip_gap);
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (FILL && hit) tasks[k + __popc(m & ((1u << lane) - 1u))] = make_int2(P, Q);
        k += __popc(m);
    }
    if (!FILL && lane == 0) counts[P] = k;
}
#endif

// ---------------------------------------------------------------------------
// Cut-off far field: one block per target particle, sweeping only the source
// particles in its neighbour list (bounding-circle gap below the cut-off);
// the block owns all its targets, so it writes complete sums. Same pair
// evaluation and masking as the chunked kernels.
// ---------------------------------------------------------------------------
#ifdef YK_DEFINE_P2P_KERNELS
template <bool MASK>
__global__ void __launch_bounds__(F32_TPB) k_p2p_f32_cut(GeomView G, const float4* __restrict__ rec,
                                                         float kscale, double skip_gap,
                                                         bool own_by_block,
                                                         const int* __restrict__ nbr_off,
                                                         const int* __restrict__ nbr,
                                                         double* __restrict__ out) {
    __shared__ float4 srcA[STILE / 2], srcB[STILE / 2];
    const int pt = blockIdx.x;
    const float kpf = (float)(LOG2E / G.rho);
    const float near_gap = 2.0f * (float)G.rho * 1.0001f + 1e-4f;
    const float short_gap = Z_SHORT * (float)G.rho, zero_gap = ZP_ZERO / kpf;
    const int n0 = nbr_off[pt], n1 = nbr_off[pt + 1];
    for (int ib = 0; ib < G.npp; ib += TPB) {
        const int l0 = ib + threadIdx.x, l1 = l0 + F32_TPB;
        const bool act0 = l0 < G.npp, act1 = l1 < G.npp;
        const int64_t ii0 = (int64_t)pt * G.npp + (act0 ? l0 : 0);
        const int64_t ii1 = (int64_t)pt * G.npp + (act1 ? l1 : 0);
        const float2 xi0 = G.xi[ii0], xi1 = G.xi[ii1];
        const int pan0 = (act0 ? l0 : 0) / G.ngl, pan1 = (act1 ? l1 : 0) / G.ngl;
        double acc0 = 0.0, acc1 = 0.0;
        for (int k = n0; k < n1; ++k) {
            const int s = nbr[k];
            const PairRange rg = block_range(G, pt, pt, s);
            if (rg.gap >= zero_gap) continue;   // every pair adds +0 in FP32
            float rc;
            const int mode = far_mode(rg, short_gap, kpf, rc);
            const PolyRZ P(mode, rc);
            TargetF32 T0, T1;
            target_setup(T0, G, pt, s, xi0, kpf, near_gap, MASK, skip_gap, pan0);
            target_setup(T1, G, pt, s, xi1, kpf, near_gap, MASK, skip_gap, pan1);
            // uniform: one target particle per block
            if ((MASK && T0.skip) || (own_by_block && T0.own)) continue;
                for (int jb = 0; jb < G.npp; jb += STILE) {
                const int cnt = min(STILE, G.npp - jb);
                const int npair = (cnt + 1) >> 1;
                __syncthreads();
                stage_rec(rec, G.npp, s, jb, cnt, srcA, srcB);
                __syncthreads();
                float r0 = 0.0f, r1 = 0.0f;
                if (!T0.close) {
                    if (mode == NARROW3) far_tile<NARROW3>(srcA, srcB, npair, T0, T1, P, r0, r1);
                else if (mode == NARROW) far_tile<NARROW>(srcA, srcB, npair, T0, T1, P, r0, r1);
                    else if (mode == FIT_SHORT)
                        far_tile<FIT_SHORT>(srcA, srcB, npair, T0, T1, P, r0, r1);
                    else far_tile<FIT_LONG>(srcA, srcB, npair, T0, T1, P, r0, r1);
                } else if (!T0.own) {
                    // close (gap <= 2 rho) implies mode FIT_LONG (gap < 10 rho)
                    const float2 TX0 = make_float2(T0.TX, T0.TX), TY0 = make_float2(T0.TY, T0.TY);
                    const float2 TX1 = make_float2(T1.TX, T1.TX), TY1 = make_float2(T1.TY, T1.TY);
                    float2 a0 = make_float2(0.0f, 0.0f), a1 = a0;
                    for (int m = 0; m < npair; ++m) {
                        const float4 A = srcA[m], B = srcB[m];
                        a0 = close2(TX0, TY0, A, B, P, a0);
                        a1 = close2(TX1, TY1, A, B, P, a1);
                    }
                    r0 = a0.x + a0.y;
                    r1 = a1.x + a1.y;
                } else {
                    for (int q = 0; q < cnt; ++q) {
                        const float4 S = src_scalar(srcA, srcB, q);
                        const int pq = (jb + q) / G.ngl;
                        if (!(T0.own && is_near_panel(T0.pan, pq, G.npan, G.near_w)))
                            r0 += PairF32::any(T0.TX - S.x, T0.TY - S.y, S.z, S.w);
                        if (!(T1.own && is_near_panel(T1.pan, pq, G.npan, G.near_w)))
                            r1 += PairF32::any(T1.TX - S.x, T1.TY - S.y, S.z, S.w);
                    }
                }
                acc0 += (double)r0;
                acc1 += (double)r1;
            }
        }
        if (act0) out[ii0] = acc0 * (double)kscale;
        if (act1) out[ii1] = acc1 * (double)kscale;
    }
}
#endif

#ifdef YK_DEFINE_P2P_KERNELS
template <bool MASK>
__global__ void __launch_bounds__(F32_TPB) k_p2p_f32_grad_cut(GeomView G,
                                                              const float4* __restrict__ rec,
                                                              double skip_gap,
                                                              const int* __restrict__ nbr_off,
                                                              const int* __restrict__ nbr,
                                                              double* __restrict__ out) {
    __shared__ float4 srcA[STILE / 2], srcB[STILE / 2];
    const int pt = blockIdx.x;
    const float kappa = (float)(1.0 / G.rho), rho = (float)G.rho;
    const float kpf = (float)(LOG2E / G.rho), inv_kp = (float)(G.rho / LOG2E);
    const float near_gap = 2.0f * (float)G.rho * 1.0001f + 1e-4f;
    const float short_gap = Z_SHORT * (float)G.rho, zero_gap = ZP_ZERO / kpf;
    const double cf = sqrt(LOG2E) * (1.0 / G.rho) * (LOG2E / G.rho);
    const int n0 = nbr_off[pt], n1 = nbr_off[pt + 1];
    for (int ib = 0; ib < G.npp; ib += TPB) {
        const int l0 = ib + threadIdx.x, l1 = l0 + F32_TPB;
        const bool act0 = l0 < G.npp, act1 = l1 < G.npp;
        const int64_t ii0 = (int64_t)pt * G.npp + (act0 ? l0 : 0);
        const int64_t ii1 = (int64_t)pt * G.npp + (act1 ? l1 : 0);
        const float2 xi0 = G.xi[ii0], xi1 = G.xi[ii1];
        const float nx0 = (float)G.nx[ii0], ny0 = (float)G.ny[ii0];
        const float nx1 = (float)G.nx[ii1], ny1 = (float)G.ny[ii1];
        const int pan0 = (act0 ? l0 : 0) / G.ngl, pan1 = (act1 ? l1 : 0) / G.ngl;
        double fast0 = 0.0, fast1 = 0.0, slow0 = 0.0, slow1 = 0.0;
        for (int k = n0; k < n1; ++k) {
            const int s = nbr[k];
            const float bg = block_range(G, pt, pt, s).gap;
            if (bg >= zero_gap) continue;   // every pair adds +0 in FP32
            const bool short_fit = bg >= short_gap;
            const PolyRZ2 P(short_fit);
            TargetF32 T0, T1;
            target_setup(T0, G, pt, s, xi0, kpf, near_gap, MASK, skip_gap, pan0);
            target_setup(T1, G, pt, s, xi1, kpf, near_gap, MASK, skip_gap, pan1);
            if (MASK && T0.skip) continue;   // uniform: one target particle per block
                for (int jb = 0; jb < G.npp; jb += STILE) {
                const int cnt = min(STILE, G.npp - jb);
                __syncthreads();
                stage_rec(rec, G.npp, s, jb, cnt, srcA, srcB);
                __syncthreads();
                float a0 = 0.0f, a1 = 0.0f, b0 = 0.0f, b1 = 0.0f;
                if (short_fit)
                    grad_tile<FIT_SHORT>(srcA, srcB, jb, cnt, G, T0, T1, true, true, nx0, ny0, nx1, ny1,
                                 inv_kp, kappa, rho, P, a0, a1, b0, b1);
                else
                    grad_tile<FIT_LONG>(srcA, srcB, jb, cnt, G, T0, T1, true, true, nx0, ny0, nx1, ny1,
                                 inv_kp, kappa, rho, P, a0, a1, b0, b1);
                fast0 += (double)a0;
                fast1 += (double)a1;
                slow0 += (double)b0;
                slow1 += (double)b1;
            }
        }
        const double sc = 1.0 / (2.0 * PI);
        if (act0) out[ii0] = (fast0 * cf + slow0) * sc;
        if (act1) out[ii1] = (fast1 * cf + slow1) * sc;
    }
}
#endif

// Cut-off neighbour lists: counts, a single-block exclusive scan, fill.
#ifdef YK_DEFINE_P2P_KERNELS
__global__ void k_nbr_count(int np, const d4* __restrict__ part, double thr, int* counts) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= np) return;
    const d4 a = part[P];
    int c = 0;
    for (int Q = 0; Q < np; ++Q) c += (Q == P || pair_in_tiles(a, part[Q], thr)) ? 1 : 0;
    counts[P] = c;
}
#endif

#ifdef YK_DEFINE_P2P_KERNELS
__global__ void k_scan_offsets(int np, const int* __restrict__ counts, int* __restrict__ off) {
    __shared__ int buf[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b = 0; b < np; b += 1024) {
        const int i = b + threadIdx.x;
        buf[threadIdx.x] = (i < np) ? counts[i] : 0;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {   // inclusive Hillis-Steele scan
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
#endif

#ifdef YK_DEFINE_P2P_KERNELS
__global__ void k_nbr_fill(int np, const d4* __restrict__ part, double thr,
                           const int* __restrict__ off, int* __restrict__ nbr) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= np) return;
    const d4 a = part[P];
    int k = off[P];
    for (int Q = 0; Q < np; ++Q)
        if (Q == P || pair_in_tiles(a, part[Q], thr)) nbr[k++] = Q;
}
#endif

// ---------------------------------------------------------------------------
// FP64 pair tiles. Value: k = K1(z)/r; the (i <- j) term is k (d . g_j) and
// the (j <- i) term is -k (d . g_i), with g = w sigma nu and d = x_i - x_j.
// Gradient: G_ij = g (nu_i . nu_j) + g' (d . nu_j)(d . nu_i)/r is symmetric;
// the terms are G_ij (w sigma)_j and G_ij (w sigma)_i.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Work item w of a launch: tile w / (npc qsplit), chunk of 256 of P's nodes
// (w / qsplit) mod npc, and the qs = w mod qsplit'th of qsplit equal ranges
// of Q's nodes. Splitting Q's nodes gives small systems, whose few tiles
// would otherwise occupy a few SMs of a GPU with a slow FP64 pipe, enough
// blocks to fill it; each item adds its partial sums to both particles.
#ifdef YK_DEFINE_P2P_KERNELS
template <bool GRAD>
__global__ void __launch_bounds__(TILE_TPB, 2) k_tiles_f64(GeomView G, const double* __restrict__ sigma,
                                                           const int2* __restrict__ tiles, int ntiles,
                                                           int qsplit, double* __restrict__ out) {
    __shared__ d4 srcQ[STILE];         // x, y, and (value) g = w sigma nu | (grad) nu
    __shared__ double wsQ[STILE];      // (grad) w sigma
    __shared__ double ys[STILE];       // Q-side sums for the staged chunk
    const double rho = G.rho, kappa = 1.0 / rho, two_rho = 2.0 * rho;
    const double scale = GRAD ? 1.0 / (2.0 * PI) : 1.0 / (2.0 * PI * rho);
    const int lane = threadIdx.x & 31;
    const int npc = (G.npp + TILE_TPB - 1) / TILE_TPB;
    const int qlen = (G.npp + qsplit - 1) / qsplit;
    const int64_t items = (int64_t)ntiles * npc * qsplit;
    for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
        const int t = (int)(w / ((int64_t)npc * qsplit));
        const int ib = (int)((w / qsplit) % npc) * TILE_TPB;
        const int q0 = (int)(w % qsplit) * qlen, q1 = min(G.npp, q0 + qlen);
        const int P = tiles[t].x, Q = tiles[t].y;
        const bool own = (P == Q);
        {
            const int li = ib + threadIdx.x;
            const bool act = li < G.npp;
            const int64_t i = (int64_t)P * G.npp + (act ? li : 0);
            const double tx = G.x[i], ty = G.y[i];
            const double tnx = G.nx[i], tny = G.ny[i];
            const double tws = act ? G.w[i] * sigma[i] : 0.0;
            const int tpan = (act ? li : 0) / G.ngl;
            double acc = 0.0;
            for (int jb = q0; jb < q1; jb += STILE) {
                const int cnt = min(STILE, q1 - jb);
                __syncthreads();
                if (threadIdx.x < cnt) {
                    const int64_t j = (int64_t)Q * G.npp + jb + threadIdx.x;
                    const double ws = G.w[j] * sigma[j];
                    if (GRAD) {
                        srcQ[threadIdx.x] = make_d4(G.x[j], G.y[j], G.nx[j], G.ny[j]);
                    } else {
                        srcQ[threadIdx.x] = make_d4(G.x[j], G.y[j], ws * G.nx[j], ws * G.ny[j]);
                    }
                    wsQ[threadIdx.x] = ws;
                    ys[threadIdx.x] = 0.0;
                }
                __syncthreads();
                for (int q = 0; q < cnt; ++q) {
                    double ki = 0.0, kj = 0.0;
                    const bool skip = own && is_near_panel(tpan, (jb + q) / G.ngl, G.npan, G.near_w);
                    if (act && !skip) {
                        const d4 S = srcQ[q];
                        const double dx = tx - S.x, dy = ty - S.y;
                        const double r2 = fma(dx, dx, dy * dy);
                        const double ri = rsqrt(r2);
                        const double z = r2 * ri * kappa;
                        if (!GRAD) {
                            double k1v;
                            if (G.eta == 0.0) {
                                if (z <= 2.0) k1v = k1_series(z);
                                else k1v = exp(-z) * p1_large(two_rho * ri) * rsqrt(z);
                            } else {   // combined representation: + eta K0 (w sigma)
                                double k0v;
                                k01(z, k0v, k1v);
                                const double sl = G.eta * rho * k0v;   // in units of 1/(2 pi rho)
                                ki = sl * wsQ[q];
                                kj = sl * tws;
                            }
                            const double k = k1v * ri;
                            ki += k * fma(dx, S.z, dy * S.w);
                            kj -= k * fma(dx, tnx * tws, dy * (tny * tws));
                        } else {
                            double k0v, k1v;
                            k01(z, k0v, k1v);
                            const double gg = k1v * ri * kappa;
                            const double gp = -(k0v * kappa + 2.0 * k1v * ri) * kappa * ri;
                            const double nn = fma(tnx, S.z, tny * S.w);
                            const double dn_s = fma(dx, S.z, dy * S.w);
                            const double dn_t = fma(dx, tnx, dy * tny);
                            const double Gij = fma(gg, nn, gp * dn_s * dn_t * ri);
                            ki = Gij * wsQ[q];
                            kj = Gij * tws;
                            if (G.eta != 0.0) {
                                // + eta nu_t . grad G: -eta K1 (d . nu_i)/(rho r) for i <- j,
                                // -eta K1 (-d . nu_j)/(rho r) for j <- i
                                const double c = G.eta * k1v * kappa * ri;
                                ki -= c * dn_t * wsQ[q];
                                kj += c * dn_s * tws;
                            }
                        }
                    }
                    acc += ki;
                    if (!own) {   // tile-uniform: the whole block takes this branch
                        const double v = warp_sum(kj);
                        if (lane == 0 && v != 0.0) atomicAdd(&ys[q], v);
                    }
                }
                if (!own) {
                    __syncthreads();
                    if (threadIdx.x < cnt)
                        atomicAdd(&out[(int64_t)Q * G.npp + jb + threadIdx.x], ys[threadIdx.x] * scale);
                }
            }
            if (act) atomicAdd(&out[i], acc * scale);
        }
    }
}
#endif

// List the particle pairs (P <= Q) with pair_in_tiles(P, Q, thr), leaving out
// P == Q when self_pairs is false (the self blocks cover them). Writes up to
// cap entries; *count receives the total.
#ifdef YK_DEFINE_P2P_KERNELS
__global__ void k_pair_list(int np, const d4* __restrict__ part, double thr, bool self_pairs,
                            int* count, int2* __restrict__ out, int cap) {
    // one warp per particle P, lanes over Q; slots reserved once per 32 Q
    const int P = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (P >= np) return;   // warp-uniform
    const d4 a = part[P];
    for (int Q0 = self_pairs ? P : P + 1; Q0 < np; Q0 += 32) {
        const int Q = Q0 + lane;
        const bool hit = Q < np && (Q == P || pair_in_tiles(a, part[Q], thr));
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (!m) continue;
        int base = 0;
        if (lane == 0) base = atomicAdd(count, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        const int k = base + __popc(m & ((1u << lane) - 1u));
        if (hit && k < cap) out[k] = make_int2(P, Q);
    }
}
#endif

// out_P (+)= S[shape(P)] sigma_P for the far part of the self block (value
// or normal derivative, FP64, or the FP32 copy for the inner operator),
// stored transposed: see k_blocks_apply.
// y_i = sum_chunks partial[c][i] + extra_i + sum_near C[shape][local i][c] sigma[near c]
__device__ __forceinline__ void assemble_at(const GeomView& G, int nchunk,
                                            const double* __restrict__ partial,
                                            const double* __restrict__ extra,
                                            const double* __restrict__ rows,
                                            const double* __restrict__ sigma,
                                            double* __restrict__ y, int64_t i) {
    if (i >= G.n) return;
    double acc = extra ? extra[i] : 0.0;
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

#ifdef YK_DEFINE_P2P_KERNELS
__global__ void k_assemble(GeomView G, int nchunk, const double* __restrict__ partial,
                           const double* __restrict__ extra, const double* __restrict__ rows,
                           const double* __restrict__ sigma, double* __restrict__ y) {
    assemble_at(G, nchunk, partial, extra, rows, sigma, y,
                blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}
#endif

// u(t) = D[sigma](t) at off-surface targets, FP64, all sources.
#ifdef YK_DEFINE_P2P_KERNELS
__global__ void __launch_bounds__(TPB) k_potential(GeomView G, const double* __restrict__ sigma,
                                                   const double* __restrict__ tgt, int64_t nt,
                                                   int ppc, double* __restrict__ partial) {
    __shared__ d4 src[STILE];
    __shared__ double wss[STILE];
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
                wss[threadIdx.x] = ws;
            }
            __syncthreads();
            if (!active) continue;
            for (int q = 0; q < cnt; ++q) {
                const d4 S = src[q];
                const double dx = tx - S.x, dy = ty - S.y;
                const double r2 = fma(dx, dx, dy * dy);
                const double ri = rsqrt(r2);
                const double z = r2 * ri * kappa;
                double k1v;
                if (G.eta == 0.0) {
                    if (z <= 2.0) k1v = k1_series(z);
                    else k1v = exp(-z) * p1_large(two_rho * ri) * rsqrt(z);
                } else {   // combined representation: + eta K0 (w sigma), units 1/(2 pi rho)
                    double k0v;
                    k01(z, k0v, k1v);
                    acc = fma(G.eta * rho * k0v, wss[q], acc);
                }
                acc = fma(k1v * ri, fma(dx, S.z, dy * S.w), acc);
            }
        }
    }
    if (active) partial[blockIdx.y * nt + i] = acc / (2.0 * PI * rho);
}
#endif

#ifdef YK_DEFINE_P2P_KERNELS
__global__ void k_sum_chunks(int64_t n, int nchunk, const double* __restrict__ partial,
                             double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int c = 0; c < nchunk; ++c) acc += partial[c * n + i];
    out[i] = acc;
}
#endif

}  // namespace yk
