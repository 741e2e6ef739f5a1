"""FP64 CPU oracle for the Stokes mobility step of the amphiphilic-particle
method (arXiv 1810.04131, Section 3: Eqs. stokes, mobility_bc, stokesjump,
mobilityu; Algorithm 1, the steps that solve for the density mu and update the
particle velocities).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import it. It shares no code with the
CUDA library; the boundary discretisation (nodes, normals, weights) is the
one of ``yk_oracle.make_geometry``, and every formula below is restated from
the paper and from the Stokes equations.

What it computes, in the paper's order:

  1. The forces and torques F_i, tau_i on the particles are given (Eq.
     mobility_bc: hydrophobic plus repulsive).
  2. The incident density sigma_inc carries them.
  3. The scattered density mu solves the boundary equation built from the
     traction jump of the stresslet (Eq. stokesjump), by a dense solve.
  4. u = S[sigma_inc + mu] on the boundaries (Eq. mobilityu, the stokeslet
     single layer), and v_i, omega_i from its averages over each boundary
     (the two formulas after Eq. mobilityu).
  5. Forward Euler (Eq. mob_vec): a_i += dt v_i, theta_i += dt omega_i.

Readings taken where the paper is silent, garbled or inconsistent:
  * Stokeslet sign: the paper prints + log|x - y| in the stokeslet. That
    kernel is not divergence free; the free-space Stokes solution is
    G = (1/(4 pi mu)) (-log r I + r r^T / r^2), r = x - y, with pressure
    p = r . f / (2 pi r^2) for a point force f. The oracle uses that.
  * Stresslet: the stress of the stokeslet flow is T_ijk = -(1/pi) r_i r_j
    r_k / r^4. It carries no viscosity (the velocity scales as 1/mu, the
    stress does not); the paper's factor 1/(pi mu) agrees at mu = 1.
  * Eq. stokesjump contracts the stresslet with the normal at the target x
    (the traction of the single layer; the printed formula drops the
    normal). With nu out of the particle into the fluid, the traction of
    S[sigma] has the limits -1/2 sigma + K* sigma from the fluid side and
    +1/2 sigma + K* sigma from inside the particle, with
    K* sigma(x) = int T(x, y) : sigma(y) nu(x) ds_y.
  * The rigid-body condition of Eq. stokes (u = v_i + omega_i (x - a_i)^perp
    on dP_i) is imposed as a vanishing traction of u = S[sigma] on the
    inside of every boundary: a Stokes flow inside P_i with zero boundary
    traction is a rigid motion, and the single layer is continuous across
    the boundary.
  * The split into incident and scattered densities: sigma_inc carries the
    given force and torque, sigma_inc = F_i / |dP_i| + tau_i (y - a_i)^perp
    / J_i with J_i = int |y - a_i|^2 ds (the normaliser of the omega formula
    after Eq. mobilityu); mu carries none. The equation for mu,
    (1/2 I + K* + W) mu = -(1/2 I + K*) sigma_inc,
    adds W, the orthogonal projector on each boundary onto the rigid motions
    (1, 0), (0, 1), (y - a_i)^perp. The range of 1/2 I + K* is orthogonal
    to the rigid motions (an interior Stokes flow exerts no net force or
    torque on its boundary), so the solution has W mu = 0: it carries no
    force or torque and solves the uncompleted equation.
  * On-surface single layer: the log singularity is integrated by product
    integration on the target's own panel and its two neighbours,
    log|x(t) - y(s)| = log|t - s| + log(|x(t) - y(s)| / |t - s|), the first
    term against the panel's Lagrange basis with exact moments, the second
    (smooth) by the Gauss-Legendre rule. The bounded r r^T / r^2 term has
    the limit tau tau^T at r = 0 and is integrated by the plain rule.
  * The traction kernel is bounded on a smooth curve: its limit at y = x is
    -(kappa / (2 pi)) tau tau^T (kappa the curvature); plain Nystrom.
  * Vectors are stored node by node (x and y component of node 0, then
    node 1, ...).
"""
from __future__ import annotations

import functools
import math
import warnings

import numpy as np
import scipy.integrate as si
import scipy.linalg as sl

from oracle.yk_oracle import make_geometry

TWO_PI = 2.0 * math.pi


# ----------------------------------------------------------------------------
# kernels
# ----------------------------------------------------------------------------

def stokeslet(r, visc=1.0):
    """G(r) (..., 2, 2) = (1/(4 pi mu)) (-log|r| I + r r^T / |r|^2)."""
    r = np.asarray(r, float)
    d2 = (r * r).sum(-1)
    G = r[..., :, None] * r[..., None, :] / d2[..., None, None]
    G = G - 0.5 * np.log(d2)[..., None, None] * np.eye(2)
    return G / (4.0 * math.pi * visc)


def stokeslet_pressure(r):
    """Pressure of the stokeslet flow per unit point force: p = r . f/(2 pi r^2),
    returned as the row vector r / (2 pi r^2) (..., 2)."""
    r = np.asarray(r, float)
    return r / (TWO_PI * (r * r).sum(-1))[..., None]


def traction_kernel(r, n_x):
    """Traction at x (normal n_x) of the stokeslet flow from y, as the 2 x 2
    matrix acting on the point force: -(1/pi) r r^T (r . n_x) / |r|^4."""
    r = np.asarray(r, float)
    d2 = (r * r).sum(-1)
    rn = (r * n_x).sum(-1)
    return -(r[..., :, None] * r[..., None, :]) * (rn / (math.pi * d2 * d2))[..., None, None]


def single_layer_blocks(logw, w, rr, visc):
    """The 2 x 2 quadrature blocks of the single layer, (N, 2, 2):
    (1/(4 pi mu)) (-logw I + w r r^T/r^2), where logw holds the weights of
    log|x - y| (product-integration weights next to the target) and rr the
    unit dyads r r^T / r^2."""
    G = -logw[:, None, None] * np.eye(2) + w[:, None, None] * rr
    return G / (4.0 * math.pi * visc)


# ----------------------------------------------------------------------------
# product integration of the logarithm
# ----------------------------------------------------------------------------

def _lagrange_basis(xk, k):
    others = np.delete(xk, k)
    den = np.prod(xk[k] - others)
    return lambda s: np.prod(s - others) / den


@functools.lru_cache(maxsize=None)
def log_moments(n_gl):
    """M[o][i][k] = int_{-1}^{1} log|xi0 - xi| L_k(xi) dxi, L_k the Lagrange
    basis of the n_gl Gauss-Legendre nodes, at xi0 = xi_i (o = 0, the
    target's own panel), xi_i + 2 (o = 1: the source panel precedes the
    target's) and xi_i - 2 (o = 2: it follows). QUADPACK's algebraic-log
    weights for xi0 inside the panel, adaptive quadrature outside."""
    xk, _ = np.polynomial.legendre.leggauss(n_gl)
    M = np.zeros((3, n_gl, n_gl))
    with warnings.catch_warnings():
        # QUADPACK notes round-off at 1e-15; the moments are checked against
        # mpmath quadrature in the tests
        warnings.simplefilter("ignore", si.IntegrationWarning)
        _fill_moments(M, xk, n_gl)
    return M


def _fill_moments(M, xk, n_gl):
    for k in range(n_gl):
        L = _lagrange_basis(xk, k)
        for i in range(n_gl):
            x0 = xk[i]
            a = si.quad(L, -1.0, x0, weight="alg-logb", wvar=(0.0, 0.0))[0]
            b = si.quad(L, x0, 1.0, weight="alg-loga", wvar=(0.0, 0.0))[0]
            M[0, i, k] = a + b
            for o, x1 in ((1, x0 + 2.0), (2, x0 - 2.0)):
                M[o, i, k] = si.quad(lambda s: math.log(abs(x1 - s)) * L(s), -1.0, 1.0,
                                     epsabs=1e-16, epsrel=1e-15, limit=400)[0]


def curvature(particles, part, t):
    """Signed curvature of x(t) = a + R(phi) (A cos t, B sin t) at each node:
    A B / (A^2 sin^2 t + B^2 cos^2 t)^(3/2) (positive: convex, counter-
    clockwise)."""
    A = particles[part, 4]
    B = particles[part, 5]
    return A * B / (A * A * np.sin(t) ** 2 + B * B * np.cos(t) ** 2) ** 1.5


# ----------------------------------------------------------------------------
# the mobility problem
# ----------------------------------------------------------------------------

class StokesOracle:
    """Boundary operators and the mobility solve for one configuration."""

    def __init__(self, particles, n_panels=16, n_gl=16, viscosity=1.0):
        self.particles = np.asarray(particles, float)
        self.geom = make_geometry(self.particles, n_panels, n_gl)
        self.visc = float(viscosity)
        g = self.geom
        self.kappa = curvature(self.particles, g.part, g.t)
        self.centre = self.particles[g.part, 1:3]
        d = g.x - self.centre
        self.e3 = np.stack([-d[:, 1], d[:, 0]], -1)          # (y - a)^perp
        npart = len(self.particles)
        self.length = np.bincount(g.part, g.w, npart)         # |dP_i|
        self.J = np.bincount(g.part, g.w * (d * d).sum(1), npart)

    @property
    def n(self):
        return self.geom.n

    # ---- operators (dense, node-major: row 2 i + c) ------------------------
    def traction_matrix(self):
        """K* (2N x 2N): K*[sigma](x_i) = sum_j w_j T(x_i - y_j, nu_i) sigma_j,
        with the diagonal limit -(kappa_i / (2 pi)) tau_i tau_i^T."""
        g = self.geom
        N = g.n
        K = np.zeros((N, 2, N, 2))
        for i in range(N):
            r = g.x[i] - g.x
            r[i] = 1.0   # placeholder, replaced below
            T = traction_kernel(r, g.nu[i]) * g.w[:, None, None]
            T[i] = -(self.kappa[i] / TWO_PI) * np.outer(g.tau[i], g.tau[i]) * g.w[i]
            K[i] = T.transpose(1, 0, 2)
        return K.reshape(2 * N, 2 * N)

    def rigid_projector(self):
        """W (2N x 2N): on each boundary the orthogonal projector (in the
        quadrature inner product) onto (1, 0), (0, 1) and (y - a)^perp."""
        g = self.geom
        N = g.n
        W = np.zeros((N, 2, N, 2))
        for p in range(len(self.particles)):
            J = np.flatnonzero(g.part == p)
            e = self.e3[J]
            blk = (np.eye(2)[None, :, None, :] / self.length[p]
                   + e[:, :, None, None] * e[None, None, :, :] / self.J[p])
            W[np.ix_(J, [0, 1], J, [0, 1])] = blk * g.w[J][None, None, :, None]
        return W.reshape(2 * N, 2 * N)

    def single_layer_matrix(self):
        """On-surface S (2N x 2N): S[sigma](x_i) = sum_j G_ij sigma_j, G of
        Eq. stokeslet with product integration of the log on the target's
        panel and its two neighbours."""
        g = self.geom
        N, ngl, npan = g.n, g.n_gl, g.n_panels
        if npan < 3:
            raise ValueError("product integration needs at least 3 panels")
        M = log_moments(ngl)
        xk, wk = np.polynomial.legendre.leggauss(ngl)
        half = math.pi / npan                                   # dt / 2
        S = np.zeros((N, 2, N, 2))
        npp = npan * ngl
        for i in range(N):
            p, P, a = g.part[i], g.panel[i], i % ngl
            r = g.x[i] - g.x
            d = np.hypot(r[:, 0], r[:, 1])
            d[i] = 1.0
            logw = g.w * np.log(d)
            rr = r[:, :, None] * r[:, None, :] / (d * d)[:, None, None]
            rr[i] = np.outer(g.tau[i], g.tau[i])
            base = p * npp
            for o, Q in ((0, P), (1, (P - 1) % npan), (2, (P + 1) % npan)):
                xi0 = xk[a] + (0.0, 2.0, -2.0)[o]
                js = base + Q * ngl + np.arange(ngl)
                dist = np.abs(xi0 - xk)                         # |t_i - s_j| / (dt/2)
                if o == 0:
                    dist[a] = 1.0
                ratio = d[js] / dist
                if o == 0:
                    ratio[a] = g.speed[i] * half                # limit of |x - y| / |xi0 - xi|
                logw[js] = g.w[js] * np.log(ratio) + half * g.speed[js] * M[o, a]
            S[i] = single_layer_blocks(logw, g.w, rr, self.visc).transpose(1, 0, 2)
        return S.reshape(2 * N, 2 * N)

    # ---- densities ----------------------------------------------------------
    def incident_density(self, F, tau):
        """sigma_inc = F_i / |dP_i| + tau_i (y - a_i)^perp / J_i on dP_i."""
        g = self.geom
        F = np.asarray(F, float).reshape(-1, 2)
        tau = np.asarray(tau, float)
        return F[g.part] / self.length[g.part, None] + \
            (tau / self.J)[g.part, None] * self.e3

    def rigid_average(self, u):
        """Eq. mobilityu's averages: v_i = int u ds / |dP_i|,
        omega_i = int (y - a_i) x u ds / J_i."""
        g = self.geom
        u = np.asarray(u, float).reshape(-1, 2)
        npart = len(self.particles)
        v = np.stack([np.bincount(g.part, g.w * u[:, 0], npart),
                      np.bincount(g.part, g.w * u[:, 1], npart)], -1) / self.length[:, None]
        om = np.bincount(g.part, g.w * (self.e3 * u).sum(1), npart) / self.J
        return v, om

    @functools.cached_property
    def operators(self):
        """(1/2 I + K*, 1/2 I + K* + W, S), built once per configuration."""
        A0 = 0.5 * np.eye(2 * self.n) + self.traction_matrix()
        return A0, A0 + self.rigid_projector(), self.single_layer_matrix()

    @functools.cached_property
    def _lu(self):
        return sl.lu_factor(self.operators[1])

    def mobility(self, F, tau):
        """The mobility problem: the velocities v (Np, 2) and angular
        velocities omega (Np,) of particles under forces F and torques tau.
        Also returns sigma = sigma_inc + mu and u = S[sigma] at the nodes."""
        A0, _, S = self.operators
        s_inc = self.incident_density(F, tau).ravel()
        mu = sl.lu_solve(self._lu, -A0 @ s_inc)
        sigma = s_inc + mu
        u = S @ sigma
        v, om = self.rigid_average(u)
        return dict(v=v, omega=om, sigma=sigma, mu=mu, u=u.reshape(-1, 2))

    def velocity(self, sigma, targets):
        """u = S[sigma] at off-surface targets (plain quadrature)."""
        g = self.geom
        s = np.asarray(sigma, float).reshape(-1, 2) * g.w[:, None]
        T = np.asarray(targets, float).reshape(-1, 2)
        out = np.zeros_like(T)
        for k, x in enumerate(T):
            out[k] = np.einsum("jab,jb->a", stokeslet(x - g.x, self.visc), s)
        return out


def mobility_step(particles, v, omega, dt):
    """Eq. mob_vec by forward Euler: a_i += dt v_i, theta_i += dt omega_i."""
    q = np.array(particles, float, copy=True)
    q[:, 1:3] += dt * np.asarray(v, float).reshape(-1, 2)
    q[:, 3] += dt * np.asarray(omega, float)
    return q
