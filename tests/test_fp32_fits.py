"""Host-side checks of the FP32 far-field kernels' constants, against scipy's
exponentially scaled Bessel function (an independent implementation):

* the K1/K0 fits the packed FP32 loops read from bessel_tables.h, in FP32
  Horner order, over the ranges the kernels use them on;
* the narrow expansions of rz^{1/2} P1(rz) about the source particle's 1/z'
  (binomial series of (1 + u)^{j+1/2}, cut after u^4 for a relative width
  up to 0.07 and after u^3 up to 0.03);
* the exact-zero skip: at z' >= 128 the largest possible pair value is below
  the smallest normal FP32 number, so ex2.approx.ftz gives +0 for every pair.
"""
import os
import re

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLES = os.path.join(ROOT, "paper_1810_04131_gb300", "csrc", "bessel_tables.h")
KERNELS = os.path.join(ROOT, "paper_1810_04131_gb300", "csrc", "p2p_kernels.cuh")
LOG2E = 1.4426950408889634


def table(name):
    txt = open(TABLES).read()
    m = re.search(r"%s\[(\d+)\] = \{([^}]*)\}" % name, txt)
    vals = [float(v.strip().rstrip("f")) for v in m.group(2).split(",")]
    assert len(vals) == int(m.group(1))
    return np.array(vals, dtype=np.float32)


def kernel_constant(name):
    m = re.search(r"constexpr float %s = ([0-9.e+-]+)f;" % name, open(KERNELS).read())
    return float(m.group(1))


def horner32(coef, x):
    acc = np.full_like(x, coef[-1], dtype=np.float32)
    for c in coef[-2::-1]:
        acc = (acc * x + np.float32(c)).astype(np.float32)
    return acc


def p_nu(nu, rz):
    """e^z z^{1/2} K_nu(z) at z = 1/(rz log2 e) (the fitted function)."""
    z = 1.0 / (rz * LOG2E)
    return scipy_special.kve(nu, z) * np.sqrt(z)


@pytest.mark.parametrize("name,nu", [("YK_P1_F32_RZ", 1), ("YK_P0_F32_RZ", 0)])
def test_packed_fits_against_scipy(name, nu):
    c = table(name)
    assert len(c) == 11
    # full fit: z >= 2 (t = 2/z in (0, 1])
    rz = np.linspace(1e-6, 1.0 / (2.0 * LOG2E), 2000).astype(np.float32)
    err = np.abs(horner32(c[:7], rz) / p_nu(nu, rz.astype(np.float64)) - 1).max()
    assert err < 2e-7, err
    # short fit: z >= 9.5
    rz = np.linspace(1e-6, 1.0 / (9.5 * LOG2E), 2000).astype(np.float32)
    err = np.abs(horner32(c[7:], rz) / p_nu(nu, rz.astype(np.float64)) - 1).max()
    assert err < 2e-7, err
    # the short fit is not good for the full range (the tables are not swapped)
    rz = np.linspace(1.0 / (4.0 * LOG2E), 1.0 / (2.0 * LOG2E), 200).astype(np.float32)
    assert np.abs(horner32(c[7:], rz) / p_nu(nu, rz.astype(np.float64)) - 1).max() > 1e-5


def binom_half(j, k):
    b = 1.0
    for i in range(k):
        b = b * (j + 0.5 - i) / (i + 1)
    return b


def test_binomial_coefficients_match_series():
    # (1 + u)^{j+1/2} = sum_k binom(j + 1/2, k) u^k, checked at small u
    for j in range(4):
        u = np.linspace(-0.07, 0.07, 41)
        series = sum(binom_half(j, k) * u ** k for k in range(30))
        assert np.allclose(series, (1 + u) ** (j + 0.5), rtol=1e-14, atol=0)


@pytest.mark.parametrize("name,degree", [("EPS_NARROW", 4), ("EPS_NARROW3", 3)])
def test_narrow_expansion_truncation(name, degree):
    eps = kernel_constant(name)
    assert 0.0 < eps <= 0.07
    p = table("YK_P1_F32_RZ")[7:].astype(np.float64)
    zshort = kernel_constant("Z_SHORT")
    worst_trunc = worst_total = 0.0
    for rc in np.geomspace(1.0 / (128 * (1 + eps)), 1.0 / (zshort * LOG2E * (1 + eps)), 300):
        a = [sum(p[j] * rc ** (j + 0.5) * binom_half(j, k) for j in range(4))
             for k in range(degree + 1)]
        rz = np.linspace(rc * (1 - eps), rc * (1 + eps), 200)
        u = rz / rc - 1
        q = sum(a[k] * u ** k for k in range(degree + 1))
        fit = np.sqrt(rz) * np.polyval(p[::-1], rz)
        worst_trunc = max(worst_trunc, np.abs(q / fit - 1).max())
        worst_total = max(worst_total, np.abs(q / (np.sqrt(rz) * p_nu(1, rz)) - 1).max())
    assert worst_trunc < 6e-8, worst_trunc
    assert worst_total < 2.5e-7, worst_total


def test_exact_zero_threshold():
    zp0 = kernel_constant("ZP_ZERO")
    assert zp0 >= 127.0
    # the true exp2(-z') at the threshold is below 2^-127; an approximation
    # with relative error 2^-22 stays below the smallest normal number 2^-126,
    # which ftz flushes to zero
    assert 2.0 ** (-zp0) * (1 + 2.0 ** -22) < 2.0 ** -126
    # a particle pair is skipped when its bounding-circle gap g has
    # g log2(e) / rho >= 128; every node pair is at least g apart
    rho = 1.0
    gap = zp0 * rho / LOG2E
    assert gap * LOG2E / rho >= zp0 - 1e-9


def test_bench_pair_classes_partition_the_interactions():
    """The bench's count of evaluated pairs by kernel mode (its roofline
    numerator) covers every far interaction between different particles
    exactly once, and uses the kernel's own thresholds."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from paper_1810_04131_gb300 import workloads as W
    assert bench.Z_SHORT == kernel_constant("Z_SHORT")
    assert bench.ZP_ZERO == kernel_constant("ZP_ZERO")
    assert np.isclose(bench.EPS_NARROW, kernel_constant("EPS_NARROW"))
    assert np.isclose(bench.EPS_NARROW3, kernel_constant("EPS_NARROW3"))
    wl = W.disks512()
    n, npp = wl.n_nodes, 256
    cls = bench.p2p_pair_classes(wl.particles, wl.rho, npp, n)
    counts = [cls[k] for k in ("full", "short", "narrow", "narrow3", "zero")]
    assert sum(counts) == n * n - wl.n_particles * npp * npp
    assert min(counts) > 0 and cls["zero"] > 0.5 * sum(counts)
    modes = {"full", "short", "narrow", "narrow3"}
    assert set(bench.FLOPS_PER_PAIR) == set(bench.LANE_OPS_PER_PAIR) == set(bench.MUFU_PER_PAIR) == modes


def bessel_i_down_f32(T, x):
    """The FMM kernels' FP32 I_0..I_T(x): the ascending series (DLMF 10.25.2)
    for the top two orders, then the downward recurrence, all in float32."""
    f = np.float32
    h = f(0.5) * f(x)
    q = h * h
    hn = f(1.0)
    for _ in range(T):
        hn = f(hn * h)
    t = f(hn * f(1.0 / np.prod(np.arange(1, T + 1, dtype=np.float64))))
    s1, s2 = t, f(T) * t
    for k in range(1, 100):
        t = f(t * f(q / (f(k) * f(T + k))))
        s1 = f(s1 + t)
        s2 = f(f(T + k) * t + s2)
        if t < f(1e-8) * s1:
            break
    I = np.zeros(T + 1, dtype=np.float32)
    I[T], I[T - 1] = s1, f(s2 / h)
    xi2 = f(2.0) / f(x)
    for k in range(T - 1, 0, -1):
        I[k - 1] = f(f(k) * xi2 * I[k] + I[k + 1])
    return I


def test_fmm_fp32_bessel_i_against_scipy():
    """The FP32 path of P2M/L2P at order 12 (I_0..I_13) is within a few FP32
    ulps of scipy's I_n for every s/rho the kernels send it (from the
    threshold below which they keep FP64 up to 3p/4 = 9), and its top term
    stays in the FP32 normal range there."""
    kern = open(os.path.join(ROOT, "paper_1810_04131_gb300", "csrc", "bessel.cuh")).read()
    xmin = float(re.search(r"BESSEL_I_F32_XMIN = ([0-9.e+-]+)f;", kern).group(1))
    T = 13
    worst = 0.0
    for x in np.geomspace(xmin, 9.0, 300):
        I = bessel_i_down_f32(T, x).astype(np.float64)
        ref = scipy_special.iv(np.arange(T + 1), x)
        worst = max(worst, float(np.max(np.abs(I / ref - 1))))
    assert worst < 2e-6, worst
    first = (0.5 * xmin) ** T / np.prod(np.arange(1, T + 1, dtype=np.float64))
    assert first > 1e-30
