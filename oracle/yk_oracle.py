"""FP64 CPU oracle for the screened-Laplace (Yukawa) double-layer Nystrom + QBX
method and its hydrophobic forces and torques (arXiv 1810.04131).

TEST INFRASTRUCTURE ONLY. This module is the slow, plain reference that the
CUDA path is checked against. Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline legs of ``bench.py`` may import it. It shares no code with
the CUDA library: Bessel functions come from scipy, quadrature rules from
numpy, and every formula is restated here from the paper.

What it computes, in the paper's order:

  1. Geometry (Section 2.1, Section 5): each particle boundary x(t) = a +
     R(phi) (A cos t, B sin t) is split into n_panels equal parameter panels
     with n_gl Gauss-Legendre nodes each (composite Gauss-Legendre panels,
     Section 6.2). nu is the unit normal out of the particle, w the
     quadrature weight times the speed |x'(t)|.
  2. Operator 1/2 I + D of Eq. (bie): the double-layer kernel
     dG/dnu_y with G = K0(|x-y|/rho)/(2 pi) (Eq. Gfunc, Eq. double-layer-def)
     by plain quadrature for far sources, and one-sided exterior QBX
     (Section 5, Eqs. local-exp, graf-coefficient, graf-addition) for the
     target's own panel and its two neighbours. The exterior expansion
     produces the jump 1/2 sigma of Eq. djump, so there is no explicit 1/2.
  3. Solve of Eq. (bie) (Algorithm 1, GMRES step): by a dense direct solve
     (the exact discrete solution) and by plain GMRES for iteration counts.
  4. Boundary gradient (Algorithm 1, step computing grad u): normal
     derivative from the same QBX expansion (near) and the gradient of the
     plain kernel (far); tangential derivative from the data f.
  5. Stress, force and torque (Eqs. stress, force_torque, scalar-torque).
  6. Off-surface potential u = D[sigma] (Eq. intrep) by plain quadrature.
  7. Optionally the combined representation of the remark on Eq. bwform:
     u = D[sigma] + eta S[sigma] (S of Eq. single-layer-def), whose
     boundary equation 1/2 sigma + D sigma + eta S sigma = f stays well
     conditioned for large rho.

Readings taken where the paper is silent (shared with the CUDA path only as
a definition, not as code):
  * K0 is the modified Bessel function of the second kind (the text says
    "first kind"; Eq. Gfunc only makes sense with K0 of the second kind).
  * QBX for Yukawa uses Graf's addition theorem for K_n and I_n:
    K0(|x-y|/rho) = sum_n K_n(|y-c|/rho) I_n(|x-c|/rho) e^{i n (theta_x - phi_y)}
    for |x-c| < |y-c| (the Yukawa form of Eq. graf-addition).
  * The double-layer expansion coefficient (the paper prints only the single
    layer one, Eq. graf-coefficient) is
    alpha_n = (1/2pi) int sigma nu_y . grad_y[K_n(s/rho) e^{-i n phi_y}] ds_y
    with (s, phi_y) the polar coordinates of y - c.
  * Expansion centre c = x + r nu, r = h/8 with h the arclength of the
    target's panel; near set = the target's panel and its two neighbours;
    QBX coefficients from those panels resampled on 8 sub-panels of n_gl
    Gauss-Legendre nodes each, with sigma interpolated panel-wise.
  * QBX order p means |n| <= p.
  * Eq. bwform writes the combined representation as i S + D for the
    Helmholtz equation with complex k. For the real screened-Laplace kernel
    the coupling is taken real and positive, u = D[sigma] + eta S[sigma],
    eta > 0: with u = 0 outside, the inside field then satisfies
    du/dnu + eta u = 0 on the boundary (jumps of Eqs. sjump and djump and of
    dS/dnu), and Green's identity makes it vanish, so the equation is
    uniquely solvable; the system stays real. The single-layer QBX
    coefficient is that of Eq. graf-coefficient in its Yukawa form,
    beta_n = (1/2pi) int sigma K_n(s/rho) e^{-i n phi_y} ds_y.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.special as sp

TWO_PI = 2.0 * math.pi

# ----------------------------------------------------------------------------
# 1. Geometry (Section 2.1 particle shapes; composite Gauss-Legendre panels)
# ----------------------------------------------------------------------------


@dataclass
class Geometry:
    particles: np.ndarray   # (Np, 6): shape, cx, cy, phi, A, B
    n_panels: int
    n_gl: int
    t: np.ndarray           # (N,) curve parameter of each node
    x: np.ndarray           # (N, 2) node positions
    nu: np.ndarray          # (N, 2) unit normal out of the particle (into water)
    tau: np.ndarray         # (N, 2) unit tangent, counter-clockwise
    speed: np.ndarray       # (N,) |x'(t)|
    w: np.ndarray           # (N,) quadrature weight (GL weight * dt/2 * speed)
    part: np.ndarray        # (N,) particle index of each node
    panel: np.ndarray       # (N,) panel index within the particle
    h: np.ndarray           # (Np, n_panels) panel arclength = sum of its weights

    @property
    def n(self):
        return self.x.shape[0]

    @property
    def n_particles(self):
        return self.particles.shape[0]


def curve(p, t):
    """Point, derivative of a particle boundary at parameter t (Section 2.1:
    ellipse with semi-axis A along the director d = (cos phi, sin phi))."""
    c, s = math.cos(p[3]), math.sin(p[3])
    A, B = p[4], p[5]
    u, v = A * np.cos(t), B * np.sin(t)
    du, dv = -A * np.sin(t), B * np.cos(t)
    x = np.stack([p[1] + c * u - s * v, p[2] + s * u + c * v], axis=-1)
    dx = np.stack([c * du - s * dv, s * du + c * dv], axis=-1)
    return x, dx


def make_geometry(particles, n_panels, n_gl):
    """Composite n_gl-point Gauss-Legendre panels, n_panels per particle."""
    particles = np.asarray(particles, dtype=np.float64)
    gx, gw = np.polynomial.legendre.leggauss(n_gl)
    dt = TWO_PI / n_panels
    k = np.arange(n_panels)
    t1 = (k[:, None] * dt + 0.5 * dt * (gx[None, :] + 1.0)).ravel()
    w1 = np.tile(0.5 * dt * gw, n_panels)
    xs, nus, taus, sps, ws, ts = [], [], [], [], [], []
    for p in particles:
        x, dx = curve(p, t1)
        spd = np.hypot(dx[:, 0], dx[:, 1])
        tau = dx / spd[:, None]
        nu = np.stack([tau[:, 1], -tau[:, 0]], axis=-1)
        xs.append(x); nus.append(nu); taus.append(tau); sps.append(spd)
        ws.append(w1 * spd); ts.append(t1)
    npp = n_panels * n_gl
    part = np.repeat(np.arange(len(particles)), npp)
    panel = np.tile(np.repeat(np.arange(n_panels), n_gl), len(particles))
    w = np.concatenate(ws)
    h = w.reshape(len(particles), n_panels, n_gl).sum(-1)
    return Geometry(particles, n_panels, n_gl, np.concatenate(ts), np.concatenate(xs),
                    np.concatenate(nus), np.concatenate(taus), np.concatenate(sps),
                    w, part, panel, h)


def label(geom, kind, param=10.0):
    """Dirichlet data f at the nodes. theta is the polar angle of x - a_i
    measured from the director d_i (Eq. JanusBC and the text after it).
    kind 0: (1 + tanh(param cos theta))/2; 1: 1 - sin^param theta;
    2: (1 + cos theta)/2."""
    a = geom.particles[geom.part, 1:3]
    phi = geom.particles[geom.part, 3]
    r = geom.x - a
    rn = np.hypot(r[:, 0], r[:, 1])
    d = np.stack([np.cos(phi), np.sin(phi)], axis=-1)
    cth = (r * d).sum(-1) / rn
    sth = (d[:, 0] * r[:, 1] - d[:, 1] * r[:, 0]) / rn
    if kind == 0:
        return 0.5 * (1.0 + np.tanh(param * cth))
    if kind == 1:
        return 1.0 - sth ** int(param)
    if kind == 2:
        return 0.5 * (1.0 + cth)
    raise ValueError("unknown label kind %r" % kind)


# ----------------------------------------------------------------------------
# 2. The layer potential
# ----------------------------------------------------------------------------


def green(x, y, rho):
    """Eq. Gfunc: G(x, y) = K0(|x - y| / rho) / (2 pi)."""
    r = np.hypot(x[..., 0] - y[..., 0], x[..., 1] - y[..., 1])
    return sp.k0(r / rho) / TWO_PI


def dl_kernel(x, y, nu_y, rho):
    """Eq. double-layer-def integrand dG(x,y)/dnu(y).

    grad_y K0(|x-y|/rho) = K1(r/rho)/rho * (x - y)/r, hence
    dG/dnu_y = K1(r/rho) ((x - y) . nu_y) / (2 pi rho r).
    """
    d0 = x[..., 0] - y[..., 0]
    d1 = x[..., 1] - y[..., 1]
    r = np.hypot(d0, d1)
    return sp.k1(r / rho) * (d0 * nu_y[..., 0] + d1 * nu_y[..., 1]) / (TWO_PI * rho * r)


def dl_kernel_grad(x, y, nu_y, rho):
    """grad_x of dG/dnu_y (for grad u = grad D[sigma]).

    With g(r) = K1(r/rho)/(rho r), the kernel is g(r) (d . nu_y)/(2 pi) with
    d = x - y, and grad_x[g (d . nu)] = g nu + g'(r) (d . nu) d / r where
    g'(r) = -(K0(r/rho)/rho + 2 K1(r/rho)/r) / (rho r)  (K1' = -K0 - K1/z).
    Returns (..., 2).
    """
    d0 = x[..., 0] - y[..., 0]
    d1 = x[..., 1] - y[..., 1]
    r = np.hypot(d0, d1)
    z = r / rho
    k0, k1 = sp.k0(z), sp.k1(z)
    g = k1 / (rho * r)
    gp = -(k0 / rho + 2.0 * k1 / r) / (rho * r)
    dn = d0 * nu_y[..., 0] + d1 * nu_y[..., 1]
    gx = (g * nu_y[..., 0] + gp * dn * d0 / r) / TWO_PI
    gy = (g * nu_y[..., 1] + gp * dn * d1 / r) / TWO_PI
    return np.stack([gx, gy], axis=-1)


def sl_kernel_grad(x, y, rho):
    """grad_x G(x, y) = -K1(r/rho) (x - y) / (2 pi rho r) (for the normal
    derivative of S[sigma]). Returns (..., 2)."""
    d0 = x[..., 0] - y[..., 0]
    d1 = x[..., 1] - y[..., 1]
    r = np.hypot(d0, d1)
    c = -sp.k1(r / rho) / (TWO_PI * rho * r)
    return np.stack([c * d0, c * d1], axis=-1)


@dataclass
class QBXParams:
    order: int = 10          # |n| <= order
    r_factor: float = 0.125  # expansion radius r = r_factor * h
    oversample: int = 8      # sub-panels per near panel
    near_width: int = 1      # neighbours on each side
    contact_factor: float = 0.5   # another particle's panel closer than this x its
                                  # arclength is integrated on its oversampled nodes


def near_panels(geom, i, near_width):
    """Panels of the target's own particle within near_width of its panel
    (cyclic). Everything else is a far source."""
    k = int(geom.panel[i])
    m = geom.n_panels
    if 2 * near_width + 1 >= m:
        return list(range(m))
    return [(k + d) % m for d in range(-near_width, near_width + 1)]


def lagrange_matrix(xc, xf):
    """Lagrange interpolation from nodes xc to points xf (rows: xf)."""
    L = np.ones((len(xf), len(xc)))
    for j in range(len(xc)):
        for k in range(len(xc)):
            if k != j:
                L[:, j] *= (xf - xc[k]) / (xc[j] - xc[k])
    return L


def lagrange_diff_matrix(xc):
    """Derivative of the Lagrange interpolant at its own nodes."""
    n = len(xc)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j:
                D[i, i] = sum(1.0 / (xc[i] - xc[k]) for k in range(n) if k != i)
            else:
                num = np.prod([xc[i] - xc[k] for k in range(n) if k not in (i, j)])
                den = np.prod([xc[j] - xc[k] for k in range(n) if k != j])
                D[i, j] = num / den
    return D


class Oracle:
    """Discrete operator of Eq. (bie) for one geometry."""

    def __init__(self, particles, n_panels=16, n_gl=16, rho=1.0, qbx=None, gamma=1.0, eta=0.0):
        self.geom = make_geometry(particles, n_panels, n_gl)
        self.rho = float(rho)
        self.gamma = float(gamma)
        # coupling of the single layer in u = D[sigma] + eta S[sigma] (0: Eq. intrep)
        self.eta = float(eta)
        self.qbx = qbx or QBXParams()
        g = self.geom
        # fine sub-panel nodes in the reference interval [-1, 1] of a panel
        xc, _ = np.polynomial.legendre.leggauss(n_gl)
        xg, wg = np.polynomial.legendre.leggauss(n_gl)
        k = self.qbx.oversample
        m = np.arange(k)
        self.fine_ref = (-1.0 + (2.0 / k) * (m[:, None] + 0.5 * (xg[None, :] + 1.0))).ravel()
        self.fine_wref = np.tile(wg / k, k)
        self.interp = lagrange_matrix(xc, self.fine_ref)      # (k*n_gl, n_gl)
        self.diff_ref = lagrange_diff_matrix(xc)               # d/dxi on [-1, 1]
        self.xc = xc

    # ---- QBX (Section 5) ---------------------------------------------------
    def qbx_centre(self, i):
        """c = x + r nu (exterior side), r = r_factor * h of the target's panel."""
        g = self.geom
        r = self.qbx.r_factor * g.h[g.part[i], g.panel[i]]
        return g.x[i] + r * g.nu[i], r

    def local_point(self, i):
        """Target i and its expansion centre in its particle's frame (centre
        at the origin, same axes): the expansion of Section 5 only involves
        positions relative to the centre c, so working in the particle frame
        avoids the rounding of world coordinates far from the origin."""
        g = self.geom
        p = g.particles[g.part[i]]
        x, _ = curve(np.array([p[0], 0.0, 0.0, p[3], p[4], p[5]]), np.array([g.t[i]]))
        r = self.qbx.r_factor * g.h[g.part[i], g.panel[i]]
        return x[0], x[0] + r * g.nu[i], r

    def fine_nodes(self, pidx, k, local=False):
        """Positions, normals and weights of the oversampled nodes of panel k
        (positions in the particle frame when local=True)."""
        g = self.geom
        dt = TWO_PI / g.n_panels
        t = k * dt + 0.5 * dt * (self.fine_ref + 1.0)
        p = g.particles[pidx]
        if local:
            p = np.array([p[0], 0.0, 0.0, p[3], p[4], p[5]])
        x, dx = curve(p, t)
        spd = np.hypot(dx[:, 0], dx[:, 1])
        nu = np.stack([dx[:, 1], -dx[:, 0]], axis=-1) / spd[:, None]
        w = 0.5 * dt * self.fine_wref * spd
        return x, nu, w

    def qbx_eval(self, i, sigma_near, want_grad=False):
        """QBX value (and normal derivative) at on-surface target i.

        sigma_near: (n_near_panels * n_gl, B) coarse density values on the
        near panels (B right-hand sides at once). Steps:
          (a) interpolate sigma from each near panel's nodes to its fine nodes;
          (b) alpha_n = (1/2pi) sum_fine w sigma nu.grad_y[K_n(s/rho) e^{-in phi}]
              for n = 0..p (alpha_{-n} = conj(alpha_n));
          (c) u = sum_{|n|<=p} alpha_n I_n(r/rho) e^{i n theta_x} at the target.
        """
        g = self.geom
        rho = self.rho
        p = self.qbx.order
        xl, c, r = self.local_point(i)
        pidx = int(g.part[i])
        panels = near_panels(g, i, self.qbx.near_width)
        ng = g.n_gl
        B = sigma_near.shape[1]
        n = np.arange(p + 2)
        alpha = np.zeros((p + 1, B), dtype=np.complex128)
        for q, k in enumerate(panels):
            y, nu, w = self.fine_nodes(pidx, k, local=True)      # (a) fine geometry
            sf = self.interp @ sigma_near[q * ng:(q + 1) * ng]    # (a) fine density
            dy = y - c
            s = np.hypot(dy[:, 0], dy[:, 1])
            phi = np.arctan2(dy[:, 1], dy[:, 0])
            es = dy / s[:, None]
            ephi = np.stack([-es[:, 1], es[:, 0]], axis=-1)
            nus = (nu * es).sum(-1)
            nuphi = (nu * ephi).sum(-1)
            Kn = sp.kv(n[:, None], (s / rho)[None, :])            # K_0..K_{p+1}
            Knp = sp.kvp(n[:p + 1, None], (s / rho)[None, :])     # K_n'
            nn = n[:p + 1, None]
            # nu . grad_y [K_n(s/rho) e^{-in phi}]
            dK = (nus[None, :] * Knp / rho - 1j * nn * nuphi[None, :] * Kn[:p + 1] / s[None, :]) \
                * np.exp(-1j * nn * phi[None, :])
            if self.eta:     # + eta K_n(s/rho) e^{-in phi}: the single layer's coefficient
                dK = dK + self.eta * Kn[:p + 1] * np.exp(-1j * nn * phi[None, :])
            alpha += (dK * w[None, :]) @ sf / TWO_PI               # (b)
        dx = xl - c
        theta = math.atan2(dx[1], dx[0])
        z = r / rho
        nn = np.arange(p + 1)
        e = np.exp(1j * nn * theta)[:, None]
        In = sp.iv(nn, z)[:, None]
        mult = np.where(nn == 0, 1.0, 2.0)[:, None]
        u = (mult * alpha * In * e).real.sum(0)                    # (c)
        if not want_grad:
            return u
        # normal derivative: the target sits at x = c - r nu, so nu . grad = -d/dr
        Inp = sp.ivp(nn, z)[:, None]
        un = -(mult * alpha * Inp * e).real.sum(0) / rho
        return u, un

    def far_kernel(self, xi, y, nu_y):
        """Kernel of the far sources: dG/dnu_y, plus eta G in the combined
        representation."""
        k = dl_kernel(xi, y, nu_y, self.rho)
        if self.eta:
            k = k + self.eta * green(xi, y, self.rho)
        return k

    def far_kernel_grad(self, xi, y, nu_y):
        """grad_x of far_kernel, (..., 2)."""
        k = dl_kernel_grad(xi, y, nu_y, self.rho)
        if self.eta:
            k = k + self.eta * sl_kernel_grad(xi, y, self.rho)
        return k

    def near_index(self, i):
        g = self.geom
        base = int(g.part[i]) * g.n_panels * g.n_gl
        panels = near_panels(g, i, self.qbx.near_width)
        return np.concatenate([base + k * g.n_gl + np.arange(g.n_gl) for k in panels])

    def far_mask(self, i):
        m = np.ones(self.geom.n, dtype=bool)
        m[self.near_index(i)] = False
        return m

    # ---- near contact: other particles' panels next to a target ----------
    def contact_panels(self, i):
        """Panels (P, k) of particles other than the target's whose nearest node
        is closer to target i than contact_factor x the panel's arclength:
        plain Gauss-Legendre quadrature on such a panel loses accuracy as the
        gap closes, so they are integrated on their oversampled nodes (the
        same 8 sub-panels and interpolation of sigma as the QBX coefficients)."""
        g = self.geom
        out = []
        cf = self.qbx.contact_factor
        if cf <= 0.0:
            return out
        ng = g.n_gl
        d = np.hypot(g.x[:, 0] - g.x[i, 0], g.x[:, 1] - g.x[i, 1])
        dmin = d.reshape(g.n_particles, g.n_panels, ng).min(-1)
        for P, k in zip(*np.nonzero(dmin < cf * g.h)):
            if P != g.part[i]:
                out.append((int(P), int(k)))
        return out

    def contact_row(self, i, P, k, want_grad=False):
        """Row entries of target i on the n_gl nodes of panel k of particle P
        by oversampled quadrature: sum_f kernel(x_i, y_f) w_f L_f(node)."""
        g = self.geom
        y, nu, w = self.fine_nodes(P, k)
        xi = g.x[i][None, :]
        kv = self.far_kernel(xi, y, nu) * w
        row = kv @ self.interp
        if not want_grad:
            return row
        kg = (self.far_kernel_grad(xi, y, nu) @ g.nu[i]) * w
        return row, kg @ self.interp

    # ---- the matvec, row by row ------------------------------------------
    def apply_rows(self, sigma, rows, want_grad=False):
        """((1/2 I + D) sigma)_i for target indices ``rows`` (and, with
        want_grad, the normal derivative of the exterior limit of D[sigma]).
        Far sources by plain quadrature, near panels by QBX."""
        g = self.geom
        sigma = np.asarray(sigma, dtype=np.float64)
        y = np.zeros(len(rows))
        yn = np.zeros(len(rows))
        for a, i in enumerate(rows):
            m = self.far_mask(i)
            xi = g.x[i][None, :]
            for P, k in self.contact_panels(i):      # oversampled instead of plain
                cols = P * g.n_panels * g.n_gl + k * g.n_gl + np.arange(g.n_gl)
                m[cols] = False
                if want_grad:
                    rv, rg = self.contact_row(i, P, k, True)
                    y[a] += rv @ sigma[cols]
                    yn[a] += rg @ sigma[cols]
                else:
                    y[a] += self.contact_row(i, P, k) @ sigma[cols]
            ws = g.w[m] * sigma[m]
            y[a] += (self.far_kernel(xi, g.x[m], g.nu[m]) * ws).sum()
            idx = self.near_index(i)
            if want_grad:
                gr = self.far_kernel_grad(xi, g.x[m], g.nu[m])
                yn[a] += ((gr @ g.nu[i]) * ws).sum()
                u, un = self.qbx_eval(i, sigma[idx][:, None], want_grad=True)
                y[a] += u[0]
                yn[a] += un[0]
            else:
                y[a] += self.qbx_eval(i, sigma[idx][:, None])[0]
        return (y, yn) if want_grad else y

    def matvec(self, sigma):
        return self.apply_rows(sigma, range(self.geom.n))

    def dense(self, want_grad=False):
        """Assemble the N x N matrix of 1/2 I + D (and of the normal
        derivative of the exterior limit). For small N only."""
        g = self.geom
        N = g.n
        A = np.zeros((N, N))
        Gn = np.zeros((N, N)) if want_grad else None
        for i in range(N):
            m = self.far_mask(i)
            xi = g.x[i][None, :]
            A[i, m] = self.far_kernel(xi, g.x[m], g.nu[m]) * g.w[m]
            idx = self.near_index(i)
            eye = np.eye(len(idx))
            if want_grad:
                Gn[i, m] = (self.far_kernel_grad(xi, g.x[m], g.nu[m]) @ g.nu[i]) * g.w[m]
            for P, k in self.contact_panels(i):      # oversampled instead of plain
                cols = P * g.n_panels * g.n_gl + k * g.n_gl + np.arange(g.n_gl)
                if want_grad:
                    A[i, cols], Gn[i, cols] = self.contact_row(i, P, k, True)
                else:
                    A[i, cols] = self.contact_row(i, P, k)
            if want_grad:
                u, un = self.qbx_eval(i, eye, want_grad=True)
                A[i, idx] = u
                Gn[i, idx] = un
            else:
                A[i, idx] = self.qbx_eval(i, eye)
        return (A, Gn) if want_grad else A

    # ---- 3. solve (Algorithm 1, GMRES step) --------------------------------
    @staticmethod
    def gmres(matvec, f, tol=1e-13, max_iter=200, x0=None):
        """Plain unrestarted GMRES: Arnoldi with modified Gram-Schmidt and a
        least-squares solve of the small Hessenberg system. Stops when
        ||f - A x|| <= tol ||f||. Returns (x, iterations, relative residual)."""
        n = len(f)
        x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
        r = f - matvec(x) if x0 is not None else f.copy()
        beta = np.linalg.norm(r)
        fn = np.linalg.norm(f)
        if fn == 0.0:
            return np.zeros(n), 0, 0.0
        if beta <= tol * fn:
            return x, 0, beta / fn
        V = np.zeros((max_iter + 1, n))
        H = np.zeros((max_iter + 1, max_iter))
        V[0] = r / beta
        rel = 1.0
        y = np.zeros(0)
        for j in range(max_iter):
            wv = matvec(V[j])
            for k in range(j + 1):
                H[k, j] = V[k] @ wv
                wv = wv - H[k, j] * V[k]
            H[j + 1, j] = np.linalg.norm(wv)
            if H[j + 1, j] > 0:
                V[j + 1] = wv / H[j + 1, j]
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)
            rel = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y) / fn
            if rel <= tol or H[j + 1, j] == 0:
                return x + V[:j + 1].T @ y, j + 1, rel
        return x + V[:max_iter].T @ y, max_iter, rel

    # ---- 4-5. gradient, stress, forces and torques --------------------------
    def tangential_derivative(self, f):
        """u_tau = df/ds on each panel: Lagrange differentiation in t
        (d/dt = (2/dt) d/dxi) divided by the speed |x'(t)|."""
        g = self.geom
        dt = TWO_PI / g.n_panels
        fp = f.reshape(-1, g.n_gl) @ self.diff_ref.T * (2.0 / dt)
        return fp.ravel() / g.speed

    def forces_torques(self, f, un):
        """Eqs. force_torque, stress, scalar-torque with grad u = u_nu nu + u_tau tau:
        T.nu = gamma [f^2/rho + rho u_tau^2 - rho u_nu^2] nu - 2 gamma rho u_nu u_tau tau.
        Returns F (Np, 2), tau (Np,) about a_i, tau0 (Np,) about the origin."""
        g = self.geom
        rho, gam = self.rho, self.gamma
        ut = self.tangential_derivative(f)
        s = gam * (f * f / rho + rho * ut * ut - rho * un * un)
        tq = -2.0 * gam * rho * un * ut
        Tn = s[:, None] * g.nu + tq[:, None] * g.tau
        wT = g.w[:, None] * Tn
        Np = g.n_particles
        F = np.zeros((Np, 2))
        np.add.at(F, g.part, wT)
        cr = g.x[:, 0] * wT[:, 1] - g.x[:, 1] * wT[:, 0]
        tau0 = np.zeros(Np)
        np.add.at(tau0, g.part, cr)
        a = g.particles[:, 1:3]
        tau = tau0 - (a[:, 0] * F[:, 1] - a[:, 1] * F[:, 0])
        return F, tau, tau0

    def energy(self, f, un):
        """Eq. main, Phi = gamma min I[u] with I[u] = int_Omega rho |grad u|^2 +
        u^2 / rho dx, in boundary form. Green's first identity on the water
        domain Omega (outward normal n = -nu on each particle boundary) with
        Delta u = u / rho^2 (Eq. SL) gives int rho |grad u|^2 = -rho int_Sigma u
        du/dnu - int u^2 / rho, so I[u] = -rho int_Sigma f du/dnu ds (u -> 0 at
        infinity). Returns the per-particle parts -gamma rho int_{Sigma_i} f u_nu ds
        (Np,); Phi is their sum."""
        g = self.geom
        e = np.zeros(g.n_particles)
        np.add.at(e, g.part, -self.gamma * self.rho * g.w * f * un)
        return e

    # ---- 6. off-surface potential (Eq. intrep) ------------------------------
    def potential(self, sigma, targets):
        g = self.geom
        t = np.asarray(targets, dtype=np.float64)
        out = np.zeros(len(t))
        ws = g.w * sigma
        for a in range(len(t)):
            out[a] = (self.far_kernel(t[a][None, :], g.x, g.nu) * ws).sum()
        return out


def closest_point(prt, tb, s0):
    """Parameter s of the boundary point of particle prt closest to tb, both
    in the particle's body frame (x(s) = (A cos s, B sin s)), by Newton's
    method on (x(s) - tb) . x'(s) = 0 started at s0."""
    A, B = prt[4], prt[5]
    s_ = s0
    for _ in range(50):
        x = np.array([A * math.cos(s_), B * math.sin(s_)])
        dx = np.array([-A * math.sin(s_), B * math.cos(s_)])
        f = (x - tb) @ dx
        fp = dx @ dx - (x - tb) @ x
        step = f / fp
        s_ -= step
        if abs(step) < 1e-15:
            break
    return s_


def _oracle_potential_near(self, sigma, targets, near_factor=1.0):
    """Eq. intrep, u = D[sigma](t), at targets anywhere in the water, also
    close to a boundary, by QBX (Section 5) for the panels near the target.

    For each particle P and target t:
      * t inside P: nan;
      * p = the boundary point of P closest to t, d = |t - p|;
      * d >= near_factor x (P's largest panel arclength): plain quadrature over
        P's nodes;
      * otherwise P's panels near p (the panel holding p +- near_width):
          - d <= 2r (r = r_factor x that panel's arclength): the local
            expansion at the target's own centre c = p + r nu(p), on the
            normal through p (so |t - c| = |d - r| <= r), with coefficients
            alpha_n from the oversampled near panels as for on-surface targets;
          - else quadrature on their oversampled nodes (sigma interpolated);
        and P's other panels by plain quadrature.
    Positions near P are taken relative to P's centre (same axes), as for the
    on-surface expansions; p itself is found in P's body frame.
    """
    g = self.geom
    rho, pq = self.rho, self.qbx.order
    t = np.asarray(targets, dtype=np.float64)
    out = np.zeros(len(t))
    ws = g.w * sigma
    ng = g.n_gl
    nn = np.arange(pq + 1)
    mult = np.where(nn == 0, 1.0, 2.0)
    dt = TWO_PI / g.n_panels
    for a in range(len(t)):
        acc = 0.0
        for P in range(g.n_particles):
            sl = np.flatnonzero(g.part == P)
            prt = g.particles[P]
            c, s_ = math.cos(prt[3]), math.sin(prt[3])
            tr = t[a] - prt[1:3]                                   # relative to the centre
            tb = np.array([c * tr[0] + s_ * tr[1], -s_ * tr[0] + c * tr[1]])   # body frame
            if (tb[0] / prt[4]) ** 2 + (tb[1] / prt[5]) ** 2 < 1.0:
                acc = np.nan
                break
            hmax = g.h[P].max()
            d2 = ((g.x[sl] - t[a]) ** 2).sum(1)
            b = int(sl[np.argmin(d2)])
            if math.sqrt(d2.min()) >= (near_factor + 1.0) * hmax:
                acc += (self.far_kernel(t[a][None, :], g.x[sl], g.nu[sl]) * ws[sl]).sum()
                continue
            sp_ = closest_point(prt, tb, g.t[b]) % TWO_PI
            pb = np.array([prt[4] * math.cos(sp_), prt[5] * math.sin(sp_)])
            tg = np.array([-prt[4] * math.sin(sp_), prt[5] * math.cos(sp_)])
            nb = np.array([tg[1], -tg[0]]) / math.hypot(*tg)
            rot = lambda v: np.array([c * v[0] - s_ * v[1], s_ * v[0] + c * v[1]])
            pt, nup = rot(pb), rot(nb)
            d = math.hypot(*(tr - pt))
            if d >= near_factor * hmax:
                acc += (self.far_kernel(t[a][None, :], g.x[sl], g.nu[sl]) * ws[sl]).sum()
                continue
            kp = int(sp_ // dt) % g.n_panels
            m = g.n_panels
            w_ = self.qbx.near_width
            panels = (list(range(m)) if 2 * w_ + 1 >= m
                      else [(kp + dd) % m for dd in range(-w_, w_ + 1)])
            near = np.isin(g.panel[sl], panels)
            far = sl[~near]
            acc += (self.far_kernel(t[a][None, :], g.x[far], g.nu[far]) * ws[far]).sum()
            sig_near = np.concatenate([sigma[sl[0] + k * ng: sl[0] + (k + 1) * ng]
                                       for k in panels])
            r = self.qbx.r_factor * g.h[P, kp]
            if d <= 2.0 * r:
                cl = pt + r * nup
                alpha = np.zeros(pq + 1, dtype=np.complex128)
                for q, k in enumerate(panels):
                    y, nu, w = self.fine_nodes(P, k, local=True)
                    sf = self.interp @ sig_near[q * ng:(q + 1) * ng]
                    dy = y - cl
                    sd = np.hypot(dy[:, 0], dy[:, 1])
                    ph = np.arctan2(dy[:, 1], dy[:, 0])
                    es = dy / sd[:, None]
                    ephi = np.stack([-es[:, 1], es[:, 0]], axis=-1)
                    nus = (nu * es).sum(-1)
                    nuphi = (nu * ephi).sum(-1)
                    Kn = sp.kv(nn[:, None], (sd / rho)[None, :])
                    Knp = sp.kvp(nn[:, None], (sd / rho)[None, :])
                    dK = (nus[None, :] * Knp / rho - 1j * nn[:, None] * nuphi[None, :] * Kn
                          / sd[None, :]) * np.exp(-1j * nn[:, None] * ph[None, :])
                    if self.eta:
                        dK = dK + self.eta * Kn * np.exp(-1j * nn[:, None] * ph[None, :])
                    alpha += (dK * (w * sf)[None, :]).sum(1) / TWO_PI
                dx = tr - cl
                rr, th = math.hypot(*dx), math.atan2(dx[1], dx[0])
                acc += (mult * alpha * sp.iv(nn, rr / rho) * np.exp(1j * nn * th)).real.sum()
            else:
                for q, k in enumerate(panels):
                    y, nu, w = self.fine_nodes(P, k, local=True)
                    sf = self.interp @ sig_near[q * ng:(q + 1) * ng]
                    acc += (self.far_kernel(tr[None, :], y, nu) * w * sf).sum()
        out[a] = acc
    return out


Oracle.potential_near = _oracle_potential_near


def solve_dense(orc, f, want_grad=True):
    """Exact discrete solution of Eq. (bie) plus u_nu, F and tau (small N)."""
    if want_grad:
        A, Gn = orc.dense(want_grad=True)
    else:
        A, Gn = orc.dense(), None
    sigma = np.linalg.solve(A, f)
    out = dict(A=A, sigma=sigma)
    if want_grad:
        un = Gn @ sigma
        F, tau, tau0 = orc.forces_torques(f, un)
        out.update(Gn=Gn, un=un, F=F, tau=tau, tau0=tau0)
    return out


# ----------------------------------------------------------------------------
# 7. Excluded-volume repulsion (Eq. repul, Section S1) and constant-drag
#    dynamics (Eq. euler; Algorithm 1 with constant drag coefficients)
# ----------------------------------------------------------------------------

def repulsion_circles(p):
    """Circle decomposition of Section S1: an ellipse (A > B) is three circles
    of radius B at a_i + k h d_i, h = A - B, k in {-1, 0, +1}; a disk is one
    circle of its radius. Returns a list per particle of (centres (n, 2),
    lever arms (n, 2), radius)."""
    out = []
    for row in np.asarray(p, float):
        shape, cx, cy, phi, A, B = row
        if int(shape) == 0 or A == B:
            out.append((np.array([[cx, cy]]), np.zeros((1, 2)), A))
        else:
            d = np.array([math.cos(phi), math.sin(phi)])
            arms = np.array([k * (A - B) * d for k in (-1, 0, 1)])
            out.append((np.array([cx, cy]) + arms, arms, B))
    return out


def repulsion(p, c0, q=3):
    """Eq. repul between every pair of circles of different particles, with
    c0 / (n_i n_j) per circle pair (n = 3 circles for an ellipse, 1 for a
    disk), so that circles recover Eq. repul exactly (the reading taken of
    Section S1's normalisation):
        f = c q / (|c_i - c_j| - (b_i + b_j))^{q+1} (c_i - c_j)/|c_i - c_j|,
    the force on particle i, its torque about a_i (lever arm x f) and the
    potential c / (|c_i - c_j| - (b_i + b_j))^q, half to each particle.
    Returns F (Np, 2), tau (Np,), phi (Np,)."""
    circ = repulsion_circles(p)
    n = len(circ)
    F = np.zeros((n, 2))
    tau = np.zeros(n)
    phi = np.zeros(n)
    for i in range(n):
        ci, ai, bi = circ[i]
        for j in range(n):
            if j == i:
                continue
            cj, _, bj = circ[j]
            c = c0 / (len(ci) * len(cj))
            for k in range(len(ci)):
                for l in range(len(cj)):
                    dvec = ci[k] - cj[l]
                    dist = math.hypot(*dvec)
                    s = dist - (bi + bj)
                    f = c * q / s ** (q + 1) * dvec / dist
                    F[i] += f
                    tau[i] += ai[k][0] * f[1] - ai[k][1] * f[0]
                    phi[i] += 0.5 * c / s ** q
    return F, tau, phi


def euler_step(p, F, tau, dt, xi_x, xi_theta):
    """Eq. euler (forward Euler with constant drag): a += dt F / xi_x,
    theta += dt tau / xi_theta, with F and tau the total (hydrophobic plus
    repulsive) force and torque."""
    q = np.array(p, float, copy=True)
    q[:, 1:3] += dt * np.asarray(F) / xi_x
    q[:, 3] += dt * np.asarray(tau) / xi_theta
    return q
