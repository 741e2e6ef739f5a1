"""Generate ``bessel_tables.h``: coefficients for the device K0/K1 routines.

Run once (needs mpmath); the generated header is committed, so building the
library needs neither this script nor mpmath.

Methods (all restated from public mathematics, not from any library):
  * z <= 2: the ascending series of DLMF 10.25.2 (I0, I1) and DLMF 10.31.1
    (K_n for n = 0, 1), with q = z^2/4:
      I0 = sum q^k / (k!)^2
      I1 = (z/2) sum q^k / (k! (k+1)!)
      K0 = -(ln(z/2) + gamma) I0 + sum_{k>=1} H_k q^k / (k!)^2
      K1 = 1/z + ln(z/2) I1 - (z/4) sum (H_k + H_{k+1} - 2 gamma) q^k / (k! (k+1)!)
    (H_k the harmonic numbers; psi(k+1) = H_k - gamma).
  * z > 2: K_nu(z) = e^{-z} z^{-1/2} P_nu(t), t = 2/z, where P_nu is a
    polynomial fitted here: Chebyshev interpolation of e^{z} sqrt(z) K_nu(z)
    (evaluated by mpmath at 40 digits) on sub-intervals of t, converted to
    monomials in the interval's local variable s in [-1, 1].
The script checks every fit against mpmath and refuses to write the header
if a fit misses its target accuracy.
"""
import os
import sys

import mpmath as mp
import numpy as np

mp.mp.dps = 40
HERE = os.path.dirname(os.path.abspath(__file__))


def p_nu(nu, t):
    z = 2 / mp.mpf(t)
    return mp.besselk(nu, z) * mp.e ** z * mp.sqrt(z)


def fit(nu, deg, a, b):
    """Chebyshev interpolant of P_nu on t in [a, b], as monomials in s."""
    n = deg + 1
    xs = [mp.cos(mp.pi * (k + mp.mpf(1) / 2) / n) for k in range(n)]
    fs = [p_nu(nu, (a + b) / 2 + (b - a) / 2 * x) for x in xs]
    c = [sum(fs[k] * mp.cos(mp.pi * j * (k + mp.mpf(1) / 2) / n) for k in range(n)) * 2 / n
         for j in range(n)]
    c[0] /= 2
    # Chebyshev -> monomial in s, in high precision
    mono = [mp.mpf(0)] * n
    tk_prev, tk = [mp.mpf(1)], [mp.mpf(0), mp.mpf(1)]
    for j in range(n):
        poly = tk_prev if j == 0 else (tk if j == 1 else None)
        if j >= 2:
            nxt = [mp.mpf(0)] * (j + 1)
            for i, v in enumerate(tk):
                nxt[i + 1] += 2 * v
            for i, v in enumerate(tk_prev):
                nxt[i] -= v
            tk_prev, tk = tk, nxt
            poly = tk
        for i, v in enumerate(poly):
            mono[i] += c[j] * v
    return [float(v) for v in mono]


def check(nu, coef, a, b, tol, dtype):
    worst = 0.0
    for t in np.linspace(max(a, 1e-6), b, 400):
        s = dtype((2 * t - (a + b)) / (b - a))
        acc = dtype(0)
        for cf in reversed(coef):
            acc = dtype(acc * s + dtype(cf))
        ref = p_nu(nu, t)
        worst = max(worst, abs(float(acc) / float(ref) - 1))
    if worst > tol:
        sys.exit("fit nu=%d [%g,%g] error %.3e > %.1e" % (nu, a, b, worst, tol))
    return worst


def series_tables(kmax):
    H = [mp.mpf(0)]
    for k in range(1, kmax + 2):
        H.append(H[-1] + mp.mpf(1) / k)
    g = mp.euler
    i0 = [1 / mp.factorial(k) ** 2 for k in range(kmax + 1)]
    i1 = [1 / (mp.factorial(k) * mp.factorial(k + 1)) for k in range(kmax + 1)]
    k0 = [H[k] / mp.factorial(k) ** 2 for k in range(kmax + 1)]
    k1 = [(H[k] + H[k + 1] - 2 * g) / (mp.factorial(k) * mp.factorial(k + 1))
          for k in range(kmax + 1)]
    return [[float(v) for v in arr] for arr in (i0, i1, k0, k1)]


def arr(name, vals, ctype="double", suffix=""):
    body = ",\n    ".join("%s%s" % (repr(float(v)), suffix) for v in vals)
    return "static __device__ __constant__ %s %s[%d] = {\n    %s};\n" % (ctype, name, len(vals), body)


def main():
    out = ["// Generated by gen_bessel_tables.py. Do not edit.",
           "// K_nu(z) = exp(-z) z^{-1/2} P(s), t = 2/z, s = (2t - (a+b))/(b-a) on t in [a, b];",
           "// Horner order: coefficient of s^0 first.",
           "#pragma once", ""]
    fits64 = [("YK_P0_FAR", 0, 12, 0.0, 0.25), ("YK_P1_FAR", 1, 12, 0.0, 0.25),
              ("YK_P0_MID", 0, 15, 0.25, 1.0), ("YK_P1_MID", 1, 15, 0.25, 1.0)]
    for name, nu, deg, a, b in fits64:
        c = fit(nu, deg, a, b)
        err = check(nu, c, a, b, 5e-16, np.float64)
        out.append("// nu=%d, t in [%g, %g], degree %d, max rel. error %.2e (FP64 Horner)" % (nu, a, b, deg, err))
        out.append(arr(name, c))
    fits32 = [("YK_P0_F32", 0, 7, 0.0, 1.0), ("YK_P1_F32", 1, 7, 0.0, 1.0)]
    for name, nu, deg, a, b in fits32:
        c = fit(nu, deg, a, b)
        err = check(nu, c, a, b, 2e-7, np.float32)
        out.append("// nu=%d, t in [%g, %g], degree %d, max rel. error %.2e (FP32 Horner)" % (nu, a, b, deg, err))
        out.append(arr(name, c, "float", "f"))
    # FP32 far field in scaled coordinates: with z' = z log2(e) and rz = 1/z',
    # t = 2/z = 2 log2(e) rz. P0, P1 as monomials in rz directly (no affine
    # step): convert the Chebyshev fit to monomials in t on [0, 1], then scale.
    for nu, name in ((1, "YK_P1_F32_RZ"), (0, "YK_P0_F32_RZ")):
        emit_rz(out, nu, name)
    kmax = 14
    return finish(out, kmax)


def rz_monomials(nu, deg, tmax):
    """Fit of P_nu on t in [0, tmax] as monomials in rz = t / (2 log2 e)."""
    from math import comb
    c = fit(nu, deg, 0.0, tmax)                    # monomial in s = (2/tmax) t - 1
    al = 2.0 / tmax
    t_mono = [0.0] * (deg + 1)
    for k, ck in enumerate(c):
        for j in range(k + 1):
            t_mono[j] += ck * comb(k, j) * (al ** j) * ((-1.0) ** (k - j))
    a = 2.0 * float(mp.log(2) ** -1)               # 2 log2(e)
    return [v * a ** j for j, v in enumerate(t_mono)], a


def rz_error(nu, rz_mono, a, tmax):
    worst = 0.0
    for t in np.linspace(1e-6, tmax, 800):
        rz = np.float32(t / a)
        acc = np.float32(rz_mono[-1])
        for cf in reversed(rz_mono[:-1]):
            acc = np.float32(acc * rz + np.float32(cf))
        worst = max(worst, abs(float(acc) / float(p_nu(nu, t)) - 1))
    return worst


def long_rz(nu):
    for deg in (6, 7):
        rz_mono, a = rz_monomials(nu, deg, 1.0)
        worst = rz_error(nu, rz_mono, a, 1.0)
        if deg == 6 and worst > 1.5e-7:
            continue
        if worst > 2e-7:
            sys.exit("rz-monomial fit error %.3e" % worst)
        return rz_mono, worst
    sys.exit("no rz-monomial fit for nu=%d" % nu)


# Short fit for particle pairs whose every node pair has z >= 10: fitted
# down to z = 9.5 (t <= 2/9.5), so that FP32 rounding of the bounding-circle
# gap that selects it stays inside the fitted range.
Z_SHORT_FIT = 9.5


def short_rz(nu):
    tmax = 2.0 / Z_SHORT_FIT
    rz_mono, a = rz_monomials(nu, 3, tmax)
    worst = rz_error(nu, rz_mono, a, tmax)
    if worst > 2e-7:
        sys.exit("short rz-monomial fit error %.3e" % worst)
    return rz_mono, worst, tmax


def emit_rz(out, nu, name):
    """One array per nu: the fit for every z > 2 (7 terms), then the short
    fit for z >= 9.5 (4 terms), so that a kernel picks either by an offset."""
    lng, e_long = long_rz(nu)
    if len(lng) != 7:
        sys.exit("the FP32 kernels expect a 7-term fit for z > 2")
    sht, e_short, tmax = short_rz(nu)
    out.append("// nu=%d in rz = 1/z' (z' = z log2 e), monomials, coefficient of rz^0 first:" % nu)
    out.append("//   [0, 7): t = 2 log2(e) rz in [0, 1] (z >= 2), degree 6, max rel. error %.2e;"
               % e_long)
    out.append("//   [7, 11): z >= %g (t in [0, %.6f]), degree 3, max rel. error %.2e (FP32 Horner)"
               % (Z_SHORT_FIT, tmax, e_short))
    out.append(arr(name, lng + sht, "float", "f"))


def finish(out, kmax):
    i0, i1, k0, k1 = series_tables(kmax)
    out.append("// ascending series (DLMF 10.25.2, 10.31.1) in q = z^2/4, k = 0..%d" % kmax)
    out.append("#define YK_SERIES_TERMS %d" % (kmax + 1))
    out.append(arr("YK_S_I0", i0))
    out.append(arr("YK_S_I1", i1))
    out.append(arr("YK_S_K0", k0))
    out.append(arr("YK_S_K1", k1))
    out.append("#define YK_SERIES_TERMS_F32 8")
    out.append(arr("YK_S_I1_F32", i1[:8], "float", "f"))
    out.append(arr("YK_S_K1_F32", k1[:8], "float", "f"))
    out.append(arr("YK_S_I0_F32", i0[:8], "float", "f"))
    out.append(arr("YK_S_K0_F32", k0[:8], "float", "f"))
    out.append("#define YK_EULER_GAMMA %r" % float(mp.euler))
    path = os.path.join(HERE, "bessel_tables.h")
    with open(path, "w") as fh:
        fh.write("\n".join(out) + "\n")
    print("wrote", path)
    return path


if __name__ == "__main__":
    main()
