"""The identities behind the FP64 particle expansions of the split operators,
checked in numpy/scipy against direct summation (no GPU).

* Graf translation for K_n: for |v| < |D|,
  K_n(|D+v|) e^{in arg(D+v)} = sum_m (-1)^m K_{n+m}(|D|) I_m(|v|) e^{i(n+m) arg D - i m arg v}.
* The double-layer potential of a particle's density, expanded about its
  centre (multipole moments M_n), translated to another particle's centre
  (local coefficients L_m) and evaluated at that particle's nodes, matches
  the direct sum of dG/dnu_y at the truncation order and band start used by
  the library (order 40, gap >= 2 bounding radii), for the value and the
  normal derivative, for smooth and for white-noise densities.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import yk_oracle as yo


def _arg(v):
    return math.atan2(v[1], v[0])


def test_graf_translation_of_K_n():
    rng = np.random.default_rng(4)
    m = np.arange(-90, 91)
    for _ in range(12):
        D = rng.normal(size=2)
        D *= rng.uniform(4.0, 9.0) / np.linalg.norm(D)
        v = rng.normal(size=2)
        v *= rng.uniform(0.1, 1.5) / np.linalg.norm(v)
        for n in (0, 1, 5, -3):
            w = D + v
            lhs = sp.kv(n, np.linalg.norm(w)) * np.exp(1j * n * _arg(w))
            rhs = ((-1.0) ** m * sp.kv(n + m, np.linalg.norm(D)) * sp.iv(m, np.linalg.norm(v))
                   * np.exp(1j * (n + m) * _arg(D) - 1j * m * _arg(v))).sum()
            assert abs(rhs - lhs) < 1e-13 * abs(lhs)


def _expand(src, tgt, sig, rho, p):
    """P2M of source particle geometry `src`, M2L to target centre, L2P at
    the target nodes (value and normal derivative), as in the library."""
    cs = src.particles[0, 1:3]
    ct = tgt.particles[0, 1:3]
    d = src.x - cs
    s = np.hypot(d[:, 0], d[:, 1])
    phi = np.arctan2(d[:, 1], d[:, 0])
    es = d / s[:, None]
    ephi = np.stack([-es[:, 1], es[:, 0]], 1)
    a_s = (src.nu * es).sum(1)
    a_p = (src.nu * ephi).sum(1)
    n = np.arange(p + 1)[:, None]
    In = sp.iv(n, s / rho)
    Inp = sp.ivp(n, s / rho)
    M = ((src.w * sig) * np.exp(-1j * n * phi) * (a_s * Inp / rho - 1j * n * a_p * In / s)).sum(1)
    Mfull = {k: (M[k] if k >= 0 else np.conj(M[-k])) for k in range(-p, p + 1)}
    D = ct - cs
    Dn, psi = np.hypot(*D), math.atan2(D[1], D[0])
    L = np.zeros(p + 1, complex)
    for mm in range(p + 1):
        L[mm] = sum(Mfull[k] * (-1) ** mm * sp.kv(k + mm, Dn / rho) * np.exp(1j * (k + mm) * psi)
                    for k in range(-p, p + 1))
    v = tgt.x - ct
    r = np.hypot(v[:, 0], v[:, 1])
    th = np.arctan2(v[:, 1], v[:, 0])
    er = v / r[:, None]
    eth = np.stack([-er[:, 1], er[:, 0]], 1)
    nr = (tgt.nu * er).sum(1)
    nt = (tgt.nu * eth).sum(1)
    m = np.arange(p + 1)[:, None]
    Im = sp.iv(m, r / rho)
    Imp = sp.ivp(m, r / rho)
    mult = np.where(m == 0, 1.0, 2.0)
    e = np.exp(-1j * m * th)
    u = (mult * (L[:, None] * e * Im)).real.sum(0) / (2 * np.pi)
    un = (mult * (L[:, None] * e * (nr * Imp / rho - 1j * m * nt * Im / r))).real.sum(0) / (2 * np.pi)
    return u, un


@pytest.mark.parametrize("rough", [False, True])
def test_particle_expansion_matches_direct_sum(rough):
    """At the band's start (a gap of 2 bounding radii) and order 40, for a
    smooth density and for white noise on the nodes (the roughest the
    discretisation carries, whose moments decay slowest)."""
    rng = np.random.default_rng(5)
    for rho, shape in ((1.0, 0), (0.25, 1), (4.0, 1)):
        A, B = (1.0, 0.5) if shape else (1.0, 1.0)
        gap = 2.0 * max(A, B) + 0.01          # the band starts at 2 bounding radii
        src = yo.make_geometry(np.array([[shape, 0.0, 0.0, 0.7, A, B]]), 16, 16)
        ang = rng.uniform(0, 2 * np.pi)
        c = (2 * max(A, B) + gap) * np.array([np.cos(ang), np.sin(ang)])
        tgt = yo.make_geometry(np.array([[shape, c[0], c[1], 2.1, A, B]]), 16, 16)
        sig = (rng.standard_normal(src.t.shape) if rough
               else 1.0 + 0.3 * np.cos(3 * src.t) + 0.2 * np.sin(src.t))
        u, un = _expand(src, tgt, sig, rho, 40)
        ws = src.w * sig
        ud = np.array([(yo.dl_kernel(x[None], src.x, src.nu, rho) * ws).sum() for x in tgt.x])
        und = np.array([((yo.dl_kernel_grad(x[None], src.x, src.nu, rho) @ nu) * ws).sum()
                        for x, nu in zip(tgt.x, tgt.nu)])
        scale = np.abs(ws).sum() * sp.k1(gap / rho) / rho + 1e-300
        assert np.abs(u - ud).max() <= 1e-13 * max(np.abs(ud).max(), scale)
        assert np.abs(un - und).max() <= 1e-12 * max(np.abs(und).max(), scale)


def _p2m(geo, sig, c, rho, p):
    """Multipole moments M_n, n = 0..p, of the double layer of `geo` about c."""
    d = geo.x - c
    s = np.hypot(d[:, 0], d[:, 1])
    phi = np.arctan2(d[:, 1], d[:, 0])
    es = d / s[:, None]
    ephi = np.stack([-es[:, 1], es[:, 0]], 1)
    a_s = (geo.nu * es).sum(1)
    a_p = (geo.nu * ephi).sum(1)
    n = np.arange(p + 1)[:, None]
    return ((geo.w * sig) * np.exp(-1j * n * phi) *
            (a_s * sp.ivp(n, s / rho) / rho - 1j * n * a_p * sp.iv(n, s / rho) / s)).sum(1)


def _full(M):
    """Coefficients -p..p from 0..p of a real field (C_{-n} = conj C_n)."""
    return np.concatenate([np.conj(M[:0:-1]), M])


def _m2m(M, t, rho, p_out):
    """Multipole about c translated to c' = c - t (t = c - c'):
    M'_k = sum_n M_n I_{k-n}(|t|/rho) e^{-i (k-n) arg t}."""
    p = len(M) - 1
    n = np.arange(-p, p + 1)[None, :]
    k = np.arange(p_out + 1)[:, None]
    return (_full(M)[None, :] * sp.iv(k - n, np.hypot(*t) / rho) *
            np.exp(-1j * (k - n) * math.atan2(t[1], t[0]))).sum(1)


def _m2l(M, D, rho, p_out):
    """Multipole about c_s to local about c_t (D = c_t - c_s):
    L_m = (-1)^m sum_n M_n K_{n+m}(|D|/rho) e^{i (n+m) arg D}."""
    p = len(M) - 1
    n = np.arange(-p, p + 1)[None, :]
    m = np.arange(p_out + 1)[:, None]
    return ((-1.0) ** m[:, 0] * (_full(M)[None, :] * sp.kv(n + m, np.hypot(*D) / rho) *
                                  np.exp(1j * (n + m) * math.atan2(D[1], D[0]))).sum(1))


def _l2l(L, s, rho, p_out):
    """Local about c to local about c'' = c + s:
    L''_j = sum_m L_m I_{m-j}(|s|/rho) e^{-i (m-j) arg s}."""
    p = len(L) - 1
    m = np.arange(-p, p + 1)[None, :]
    j = np.arange(p_out + 1)[:, None]
    return (_full(L)[None, :] * sp.iv(m - j, np.hypot(*s) / rho) *
            np.exp(-1j * (m - j) * math.atan2(s[1], s[0]))).sum(1)


def _l2p(L, c, x, rho):
    """u(x) = (1/2pi) sum_m L_m I_m(|x-c|/rho) e^{-i m arg(x-c)} (real field)."""
    v = x - c
    r = np.hypot(v[:, 0], v[:, 1])
    th = np.arctan2(v[:, 1], v[:, 0])
    m = np.arange(len(L))[:, None]
    mult = np.where(m == 0, 1.0, 2.0)
    return (mult * L[:, None] * sp.iv(m, r / rho) * np.exp(-1j * m * th)).real.sum(0) / (2 * np.pi)


def test_m2m_matches_direct_moments():
    """Translating the moments about a particle's centre to another centre
    reproduces the moments computed there directly (the I_n addition theorem
    is exact; only the source order truncates)."""
    rng = np.random.default_rng(11)
    for rho, shape in ((1.0, 0), (0.5, 1), (4.0, 1)):
        A, B = (1.0, 0.5) if shape else (1.0, 1.0)
        geo = yo.make_geometry(np.array([[shape, 0.3, -0.2, 1.1, A, B]]), 16, 16)
        sig = 1.0 + 0.3 * np.cos(3 * geo.t) + 0.2 * rng.standard_normal(geo.t.shape)
        c = geo.particles[0, 1:3]
        for t in (np.array([1.5, -2.0]), np.array([-3.0, 0.7])):
            M = _p2m(geo, sig, c, rho, 70)
            M2 = _m2m(M, t, rho, 12)
            ref = _p2m(geo, sig, c - t, rho, 12)
            assert np.abs(M2 - ref).max() <= 1e-12 * np.abs(ref).max()


def test_l2l_matches_parent_expansion():
    """A local expansion shifted to a child centre takes the same values
    near that centre."""
    rng = np.random.default_rng(12)
    for rho in (0.5, 1.0, 4.0):
        L = (rng.standard_normal(61) + 1j * rng.standard_normal(61)) * 0.5 ** np.arange(61)
        L[0] = L[0].real
        s = np.array([1.2, -0.9])
        Lc = _l2l(L, s, rho, 60)
        x = s + rng.uniform(-0.7, 0.7, size=(20, 2))
        u0 = _l2p(L, np.zeros(2), x, rho)
        u1 = _l2p(Lc, s, x, rho)
        assert np.abs(u1 - u0).max() <= 1e-12 * np.abs(u0).max()


def test_fmm_chain_matches_direct_sum():
    """P2M about a leaf centre, M2M to the parent, M2L between parents,
    L2L to a child, L2P at another particle's nodes: the chain the quadtree
    FMM runs equals the direct double-layer sum. At order 30 it is exact to
    rounding; at order 12 (the default of the FMM far field) the error is
    bounded by 1e-7 of the source strength at this separation."""
    rng = np.random.default_rng(13)
    for rho, shape in ((1.0, 0), (4.0, 1)):
        A, B = (1.0, 0.5) if shape else (1.0, 1.0)
        # leaf side b; source leaf [0, b]^2 in parent [0, 2b]^2; target leaf
        # [4b, 5b] x [0, b] in parent [4b, 6b] x [0, 2b]: the parents are one
        # box apart, the closest pair an FMM interaction list holds
        b = 8.0
        src = yo.make_geometry(np.array([[shape, 2.5, 1.0, 0.4, A, B]]), 16, 16)
        tgt = yo.make_geometry(np.array([[shape, 36.0, 5.0, 2.0, A, B]]), 16, 16)
        sig = 1.0 + 0.3 * np.cos(3 * src.t) + 0.2 * rng.standard_normal(src.t.shape)
        c_leaf_s, c_par_s = np.array([b / 2, b / 2]), np.array([b, b])
        c_par_t, c_leaf_t = np.array([5 * b, b]), np.array([4.5 * b, b / 2])
        ws = src.w * sig
        ud = np.array([(yo.dl_kernel(x[None], src.x, src.nu, rho) * ws).sum() for x in tgt.x])
        for p, tol in ((30, 1e-13), (12, 1e-7)):
            M = _m2m(_p2m(src, sig, c_leaf_s, rho, p), c_leaf_s - c_par_s, rho, p)
            L = _m2l(M, c_par_t - c_par_s, rho, p)
            L = _l2l(L, c_leaf_t - c_par_t, rho, p)
            u = _l2p(L, c_leaf_t, tgt.x, rho)
            assert np.abs(u - ud).max() <= tol * np.abs(ws).sum() + 1e-14 * np.abs(ud).max()
