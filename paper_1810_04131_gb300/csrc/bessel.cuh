// Device modified Bessel functions for the Yukawa kernel G = K0(r/rho)/(2 pi)
// (Eq. Gfunc) and its QBX expansions (Section 5, Graf addition for K_n, I_n).
//
// K0, K1 (FP64 and FP32):
//   z <= 2  ascending series, DLMF 10.25.2 and 10.31.1 (coefficients in
//           bessel_tables.h, generated from exact rationals);
//   z > 2   K_nu(z) = exp(-z) z^{-1/2} P_nu(t), t = 2/z, with P_nu a
//           project-fitted polynomial (gen_bessel_tables.py, Chebyshev
//           interpolation of exp(z) sqrt(z) K_nu(z), checked to 2.2e-16 in FP64
//           and 1e-7 in FP32).
// K_n for n >= 2: forward recurrence K_{n+1} = K_{n-1} + (2n/z) K_n
// (DLMF 10.29.1), stable for K. I_n: ascending series DLMF 10.25.2.
#pragma once
#include "bessel_tables.h"

namespace yk {

template <int NT>
__device__ __forceinline__ double horner(const double (&c)[NT], double s) {
    double acc = c[NT - 1];
#pragma unroll
    for (int k = NT - 2; k >= 0; --k) acc = fma(acc, s, c[k]);
    return acc;
}

template <int NT>
__device__ __forceinline__ float hornerf(const float (&c)[NT], float s) {
    float acc = c[NT - 1];
#pragma unroll
    for (int k = NT - 2; k >= 0; --k) acc = fmaf(acc, s, c[k]);
    return acc;
}

// ---- FP64 ------------------------------------------------------------------

// K0 and K1 for z <= 2 (series).
__device__ __forceinline__ void k01_series(double z, double& k0, double& k1) {
    const double q = 0.25 * z * z;
    double si0 = YK_S_I0[YK_SERIES_TERMS - 1], si1 = YK_S_I1[YK_SERIES_TERMS - 1];
    double sk0 = YK_S_K0[YK_SERIES_TERMS - 1], sk1 = YK_S_K1[YK_SERIES_TERMS - 1];
#pragma unroll
    for (int k = YK_SERIES_TERMS - 2; k >= 0; --k) {
        si0 = fma(si0, q, YK_S_I0[k]);
        si1 = fma(si1, q, YK_S_I1[k]);
        sk0 = fma(sk0, q, YK_S_K0[k]);
        sk1 = fma(sk1, q, YK_S_K1[k]);
    }
    const double lg = log(0.5 * z);
    k0 = -(lg + YK_EULER_GAMMA) * si0 + sk0;  // the k = 0 coefficient H_0 is zero
    k1 = 1.0 / z + lg * (0.5 * z) * si1 - 0.25 * z * sk1;
}

// K1 alone for z <= 2 (series).
__device__ __forceinline__ double k1_series(double z) {
    const double q = 0.25 * z * z;
    double si1 = YK_S_I1[YK_SERIES_TERMS - 1], sk1 = YK_S_K1[YK_SERIES_TERMS - 1];
#pragma unroll
    for (int k = YK_SERIES_TERMS - 2; k >= 0; --k) {
        si1 = fma(si1, q, YK_S_I1[k]);
        sk1 = fma(sk1, q, YK_S_K1[k]);
    }
    return 1.0 / z + log(0.5 * z) * (0.5 * z) * si1 - 0.25 * z * sk1;
}

// exp(z) sqrt(z) K_nu(z) for z > 2, nu = 0, 1 (polynomial in t = 2/z).
__device__ __forceinline__ double p1_large(double t) {
    if (t <= 0.25) return horner(YK_P1_FAR, 8.0 * t - 1.0);
    return horner(YK_P1_MID, (2.0 * t - 1.25) * (1.0 / 0.75));
}
__device__ __forceinline__ double p0_large(double t) {
    if (t <= 0.25) return horner(YK_P0_FAR, 8.0 * t - 1.0);
    return horner(YK_P0_MID, (2.0 * t - 1.25) * (1.0 / 0.75));
}

// K1(z), z > 0.
__device__ __forceinline__ double k1(double z) {
    if (z <= 2.0) return k1_series(z);
    return exp(-z) * p1_large(2.0 / z) * rsqrt(z);
}

// K0(z), K1(z), z > 0.
__device__ __forceinline__ void k01(double z, double& k0, double& k1) {
    if (z <= 2.0) {
        k01_series(z, k0, k1);
        return;
    }
    const double t = 2.0 / z;
    const double e = exp(-z) * rsqrt(z);
    k0 = e * p0_large(t);
    k1 = e * p1_large(t);
}

// 1/d for an integer-valued d in [1, 2^24): the FP32 rcp.approx estimate
// refined by two Newton-Raphson steps r <- r + r (1 - d r) (each step
// doubles the number of correct bits: 2^-23 -> 2^-46 -> FP64 rounding).
__device__ __forceinline__ double recip_int(double d) {
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"((float)d));
    double r = (double)rf;
    r = fma(r, fma(-d, r, 1.0), r);
    return fma(r, fma(-d, r, 1.0), r);
}

// 1/n! for n = 0..63 (constant-initialised at compile time)
constexpr double inv_fact_c(int n) {
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r /= k;
    return r;
}
#define YK_IF4(n) inv_fact_c(n), inv_fact_c(n + 1), inv_fact_c(n + 2), inv_fact_c(n + 3)
static __constant__ double c_inv_fact[64] = {
    YK_IF4(0),  YK_IF4(4),  YK_IF4(8),  YK_IF4(12), YK_IF4(16), YK_IF4(20), YK_IF4(24), YK_IF4(28),
    YK_IF4(32), YK_IF4(36), YK_IF4(40), YK_IF4(44), YK_IF4(48), YK_IF4(52), YK_IF4(56), YK_IF4(60)};
#undef YK_IF4

// I_n(x) and I_{n-1}(x), 1 <= n <= 63, from one ascending series (DLMF 10.25.2):
// with t_k = (x/2)^{n+2k} / (k! (n+k)!), I_n = sum t_k and
// I_{n-1} = (2/x) sum (n+k) t_k.
__device__ inline void bessel_i_pair(int n, double x, double& In, double& In1) {
    const double h = 0.5 * x, q = h * h;
    double hn = 1.0;
    for (int k = 0; k < n; ++k) hn *= h;
    double t = hn * c_inv_fact[n];
    double s1 = t, s2 = n * t;
    for (int k = 1; k < 200; ++k) {
        t *= q * recip_int((double)k * (double)(n + k));
        s1 += t;
        s2 = fma((double)(n + k), t, s2);
        if (t < 1e-17 * s1) break;
    }
    In = s1;
    In1 = s2 / h;
}

// I_0..I_top(x), 1 <= top <= 63, x > 0: the top two orders from the series,
// then the backward recurrence I_{k-1} = I_{k+1} + (2k/x) I_k (stable
// downwards).
__device__ inline void bessel_i_down(int top, double x, double* I) {
    bessel_i_pair(top, x, I[top], I[top - 1]);
    const double xi2 = 2.0 / x;
    for (int k = top - 1; k >= 1; --k) I[k - 1] = fma(k * xi2, I[k], I[k + 1]);
}

// I_n(z) for n = 0..nmax (ascending series, DLMF 10.25.2); small to moderate z.
__device__ inline double bessel_i_series(int n, double z) {
    const double q = 0.25 * z * z;
    double term = 1.0;
    for (int k = 1; k <= n; ++k) term *= (0.5 * z) / k;  // (z/2)^n / n!
    double sum = term;
    for (int k = 1; k < 200; ++k) {
        term *= q / ((double)k * (double)(n + k));
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

// ---- FP32 ------------------------------------------------------------------

// I_0..I_T(x) in FP32 for a fixed top order T (so that I stays in
// registers): I_T and I_{T-1} from the ascending series (DLMF 10.25.2) as in
// bessel_i_pair, then the downward recurrence I_{k-1} = I_{k+1} + (2k/x) I_k.
// For T <= 13 and x >= BESSEL_I_F32_XMIN the series' first term
// (x/2)^T / T! stays above 1e-30, inside the FP32 normal range.
constexpr float BESSEL_I_F32_XMIN = 0.06f;
template <int T>
__device__ __forceinline__ void bessel_i_down_f(float x, float (&I)[T + 1]) {
    static_assert(T >= 1 && T <= 13, "order range of the FP32 series");
    const float h = 0.5f * x, q = h * h;
    float hn = 1.0f;
#pragma unroll
    for (int k = 0; k < T; ++k) hn *= h;
    float t = hn * (float)c_inv_fact[T];
    float s1 = t, s2 = (float)T * t;
    for (int k = 1; k < 100; ++k) {
        t *= q / ((float)k * (float)(T + k));
        s1 += t;
        s2 = fmaf((float)(T + k), t, s2);
        if (t < 1e-8f * s1) break;
    }
    I[T] = s1;
    I[T - 1] = s2 / h;
    const float xi2 = 2.0f / x;
#pragma unroll
    for (int k = T - 1; k >= 1; --k) I[k - 1] = fmaf((float)k * xi2, I[k], I[k + 1]);
}

// K1(z) in FP32; rinv_rho2 = t = 2/z supplied by the caller (it has 1/r).
__device__ __forceinline__ float k1f(float z, float t) {
    if (z > 2.0f) {
        return __expf(-z) * hornerf(YK_P1_F32, 2.0f * t - 1.0f) * sqrtf(0.5f * t);
    }
    const float q = 0.25f * z * z;
    float si1 = YK_S_I1_F32[YK_SERIES_TERMS_F32 - 1], sk1 = YK_S_K1_F32[YK_SERIES_TERMS_F32 - 1];
#pragma unroll
    for (int k = YK_SERIES_TERMS_F32 - 2; k >= 0; --k) {
        si1 = fmaf(si1, q, YK_S_I1_F32[k]);
        sk1 = fmaf(sk1, q, YK_S_K1_F32[k]);
    }
    return 0.5f * t + logf(0.5f * z) * (0.5f * z) * si1 - 0.25f * z * sk1;
}

// K0, K1 in FP32.
__device__ __forceinline__ void k01f(float z, float t, float& k0, float& k1) {
    if (z > 2.0f) {
        const float e = __expf(-z) * sqrtf(0.5f * t);
        const float s = 2.0f * t - 1.0f;
        k0 = e * hornerf(YK_P0_F32, s);
        k1 = e * hornerf(YK_P1_F32, s);
        return;
    }
    const float q = 0.25f * z * z;
    float si0 = YK_S_I0_F32[YK_SERIES_TERMS_F32 - 1], si1 = YK_S_I1_F32[YK_SERIES_TERMS_F32 - 1];
    float sk0 = YK_S_K0_F32[YK_SERIES_TERMS_F32 - 1], sk1 = YK_S_K1_F32[YK_SERIES_TERMS_F32 - 1];
#pragma unroll
    for (int k = YK_SERIES_TERMS_F32 - 2; k >= 0; --k) {
        si0 = fmaf(si0, q, YK_S_I0_F32[k]);
        si1 = fmaf(si1, q, YK_S_I1_F32[k]);
        sk0 = fmaf(sk0, q, YK_S_K0_F32[k]);
        sk1 = fmaf(sk1, q, YK_S_K1_F32[k]);
    }
    const float lg = logf(0.5f * z);
    k0 = -(lg + (float)YK_EULER_GAMMA) * si0 + sk0;
    k1 = 0.5f * t + lg * (0.5f * z) * si1 - 0.25f * z * sk1;
}

}  // namespace yk
