"""The identities behind the FP64 particle expansions of the split operators,
checked in numpy/scipy against direct summation (no GPU).

* Graf translation for K_n: for |v| < |D|,
  K_n(|D+v|) e^{in arg(D+v)} = sum_m (-1)^m K_{n+m}(|D|) I_m(|v|) e^{i(n+m) arg D - i m arg v}.
* The double-layer potential of a particle's density, expanded about its
  centre (multipole moments M_n), translated to another particle's centre
  (local coefficients L_m) and evaluated at that particle's nodes, matches
  the direct sum of dG/dnu_y at the truncation order and band start used by
  the library (order 40, gap >= 4 bounding radii), for the value and the
  normal derivative.
"""
import math

import numpy as np
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


def test_particle_expansion_matches_direct_sum():
    rng = np.random.default_rng(5)
    for rho, shape in ((1.0, 0), (0.25, 1), (4.0, 1)):
        A, B = (1.0, 0.5) if shape else (1.0, 1.0)
        gap = 4.0 * max(A, B) + 0.01          # the band starts at 4 bounding radii
        src = yo.make_geometry(np.array([[shape, 0.0, 0.0, 0.7, A, B]]), 16, 16)
        ang = rng.uniform(0, 2 * np.pi)
        c = (2 * max(A, B) + gap) * np.array([np.cos(ang), np.sin(ang)])
        tgt = yo.make_geometry(np.array([[shape, c[0], c[1], 2.1, A, B]]), 16, 16)
        sig = 1.0 + 0.3 * np.cos(3 * src.t) + 0.2 * np.sin(src.t)
        u, un = _expand(src, tgt, sig, rho, 40)
        ws = src.w * sig
        ud = np.array([(yo.dl_kernel(x[None], src.x, src.nu, rho) * ws).sum() for x in tgt.x])
        und = np.array([((yo.dl_kernel_grad(x[None], src.x, src.nu, rho) @ nu) * ws).sum()
                        for x, nu in zip(tgt.x, tgt.nu)])
        scale = np.abs(ws).sum() * sp.k1(gap / rho) / rho + 1e-300
        assert np.abs(u - ud).max() <= 1e-13 * max(np.abs(ud).max(), scale)
        assert np.abs(un - und).max() <= 1e-12 * max(np.abs(und).max(), scale)
