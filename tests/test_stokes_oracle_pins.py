"""Pins of the Stokes mobility oracle (oracle/stokes_oracle.py; Section 3,
Eqs. stokes, mobility_bc, stokesjump, mobilityu) against what the Stokes
equations and closed forms fix, not against the oracle's own formulas:

  * kernels: the stokeslet flow is divergence free and balances its pressure
    (mu Lap u = grad p, centered differences); the traction kernel is the
    stress of that flow contracted with the normal (centered differences);
    the traction through a circle around a unit point force is -f;
  * log moments: exact on polynomials against mpmath quadrature;
  * on-surface single layer: closed forms on a circle (mean value of the log,
    the rotlet, S[nu] = 0 by incompressibility) and adaptive quadrature of
    the continuous integral on an ellipse;
  * traction operator: K*[nu] = nu/2 on any closed curve (the pressure jump
    of S[nu]); K*[e] = -e/2 and K*[tau] = -tau/2 on a circle (uniform flow
    and rigid rotation inside); its range carries no force or torque;
    adaptive quadrature on an ellipse;
  * mobility: a single disk under a torque (rotlet) and a force (closed
    form); several particles: the boundary velocity is a rigid motion, the
    density carries the given force and torque, the mobility matrix is
    symmetric (Lorentz reciprocity) and positive on force- and torque-free
    loads (Eq. energy_dissipation), the point-force limit of two distant
    disks, convergence under panel refinement;
  * planted mistakes in the oracle are caught by these pins.
"""
import math
import warnings

import numpy as np
import pytest
import scipy.integrate as si

from oracle import stokes_oracle as so

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")

DISK, ELLIPSE = 0, 1


def _disk(a=1.0, cx=0.3, cy=-0.2, phi=0.4):
    return np.array([[DISK, cx, cy, phi, a, a]])


def _three():
    return np.array([[DISK, 0.0, 0.0, 0.3, 1.0, 1.0],
                     [ELLIPSE, 2.6, 0.4, 1.1, 1.0, 0.5],
                     [DISK, 0.5, 2.5, 2.0, 0.8, 0.8]])


# --------------------------------------------------------------------------
# kernels
# --------------------------------------------------------------------------

def _u(x, f, mu):
    return so.stokeslet(x, mu) @ f


def test_stokeslet_is_a_stokes_flow():
    rng = np.random.default_rng(0)
    mu = 1.7
    for _ in range(5):
        x = rng.uniform(-2, 2, 2)
        x *= 0.5 + rng.random() / np.linalg.norm(x)
        f = rng.standard_normal(2)
        h = 1e-4
        ex, ey = np.array([h, 0.0]), np.array([0.0, h])
        div = ((_u(x + ex, f, mu) - _u(x - ex, f, mu))[0]
               + (_u(x + ey, f, mu) - _u(x - ey, f, mu))[1]) / (2 * h)
        assert abs(div) < 1e-8
        h = 5e-4
        ex, ey = np.array([h, 0.0]), np.array([0.0, h])
        lap = (_u(x + ex, f, mu) + _u(x - ex, f, mu) + _u(x + ey, f, mu) + _u(x - ey, f, mu)
               - 4 * _u(x, f, mu)) / h ** 2
        p = lambda y: so.stokeslet_pressure(y) @ f
        gp = np.array([p(x + ex) - p(x - ex), p(x + ey) - p(x - ey)]) / (2 * h)
        assert np.abs(mu * lap - gp).max() < 2e-6 * np.abs(gp).max()


def test_traction_kernel_is_the_stress_of_the_stokeslet():
    rng = np.random.default_rng(1)
    mu = 0.6
    h = 1e-5
    for _ in range(5):
        x = rng.uniform(-2, 2, 2)
        f = rng.standard_normal(2)
        n = rng.standard_normal(2)
        n /= np.linalg.norm(n)
        grad = np.zeros((2, 2))   # grad[i, k] = d u_i / d x_k
        for k in range(2):
            e = np.zeros(2)
            e[k] = h
            grad[:, k] = (_u(x + e, f, mu) - _u(x - e, f, mu)) / (2 * h)
        p = so.stokeslet_pressure(x) @ f
        stress = -p * np.eye(2) + mu * (grad + grad.T)
        t = so.traction_kernel(x, n) @ f
        assert np.abs(stress @ n - t).max() < 1e-7 * np.abs(t).max() + 1e-9


def test_traction_through_a_circle_is_minus_the_point_force():
    f = np.array([0.7, -1.3])
    for R in (0.5, 3.0):
        th = np.linspace(0, 2 * math.pi, 64, endpoint=False)
        n = np.stack([np.cos(th), np.sin(th)], -1)
        t = so.traction_kernel(R * n, n) @ f
        assert np.abs(t.sum(0) * R * 2 * math.pi / 64 + f).max() < 1e-14


# --------------------------------------------------------------------------
# product integration of the logarithm
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n_gl", [7, 16])
def test_log_moments_are_exact_on_polynomials(n_gl):
    import mpmath as mp
    mp.mp.dps = 30
    M = so.log_moments(n_gl)
    xk, _ = np.polynomial.legendre.leggauss(n_gl)
    for i in (0, n_gl // 2, n_gl - 1):
        for o, shift in ((0, 0.0), (1, 2.0), (2, -2.0)):
            x0 = xk[i] + shift
            for m in range(4):
                pts = [-1, x0, 1] if o == 0 else [-1, 1]
                ref = float(mp.quad(lambda s: mp.log(abs(mp.mpf(x0) - s)) * s ** m, pts))
                assert abs(M[o, i] @ xk ** m - ref) < 2e-15, (o, i, m)


# --------------------------------------------------------------------------
# on-surface single layer
# --------------------------------------------------------------------------

@pytest.mark.parametrize("a,mu", [(1.0, 1.0), (2.5, 2.0)])
def test_single_layer_on_a_circle(a, mu):
    """S[e] = a (1 - 2 log a) e / (4 mu) (mean of log|x - y| over the circle
    is log a, mean of r r^T / r^2 is I/2); S[tau] = a tau / (2 mu) (the
    rotlet of torque 2 pi a^2 at radius a); S[nu] = 0 (incompressibility)."""
    o = so.StokesOracle(_disk(a), 16, 16, mu)
    S = o.operators[2]
    g = o.geom
    e = np.tile([0.6, -0.8], g.n)
    assert np.abs(S @ e - a * (1 - 2 * math.log(a)) / (4 * mu) * e).max() < 1e-13
    t = g.tau.ravel()
    assert np.abs(S @ t - a / (2 * mu) * t).max() < 1e-13
    assert np.abs(S @ g.nu.ravel()).max() < 1e-13


def _ellipse_curve(A, B, phi, c):
    R = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
    def pos(t):
        return c + R @ np.array([A * math.cos(t), B * math.sin(t)])
    def der(t):
        return R @ np.array([-A * math.sin(t), B * math.cos(t)])
    return pos, der


def _density(t):
    return np.array([math.cos(t) + 0.3 * math.sin(2 * t), 0.5 - math.sin(t)])


def test_single_layer_brute_force_on_an_ellipse():
    A, B, phi, c = 1.3, 0.6, 0.7, np.array([0.4, -0.1])
    p = np.array([[ELLIPSE, c[0], c[1], phi, A, B]])
    o = so.StokesOracle(p, 16, 16, 1.3)
    g = o.geom
    sig = np.array([_density(t) for t in g.t]).ravel()
    u = (o.operators[2] @ sig).reshape(-1, 2)
    pos, der = _ellipse_curve(A, B, phi, c)
    for i in (0, 37, 130, 255):
        ti = g.t[i]
        ref = np.zeros(2)
        for comp in range(2):
            def f(s):
                return (so.stokeslet(g.x[i] - pos(s), 1.3) @ _density(s))[comp] * \
                    np.linalg.norm(der(s))
            ref[comp] = sum(si.quad(f, a, b, limit=400, epsabs=1e-15, epsrel=1e-14)[0]
                            for a, b in ((ti - math.pi, ti), (ti, ti + math.pi)))
        assert np.abs(u[i] - ref).max() < 1e-12, (i, u[i] - ref)


# --------------------------------------------------------------------------
# traction operator
# --------------------------------------------------------------------------

def test_traction_identities():
    for p in (_disk(1.7), np.array([[ELLIPSE, 1.0, 2.0, 0.3, 1.0, 0.5]])):
        o = so.StokesOracle(p, 16, 16)
        K = o.operators[0] - 0.5 * np.eye(2 * o.n)
        n = o.geom.nu.ravel()
        assert np.abs(K @ n - 0.5 * n).max() < 1e-12
    o = so.StokesOracle(_disk(1.7), 16, 16)
    K = o.operators[0] - 0.5 * np.eye(2 * o.n)
    e = np.tile([0.3, 1.1], o.n)
    t = o.geom.tau.ravel()
    assert np.abs(K @ e + 0.5 * e).max() < 1e-12
    assert np.abs(K @ t + 0.5 * t).max() < 1e-12


def test_interior_traction_carries_no_force_or_torque():
    o = so.StokesOracle(_three(), 16, 16)
    g = o.geom
    sig = np.random.default_rng(3).standard_normal(2 * o.n)
    t = (o.operators[0] @ sig).reshape(-1, 2)
    scale = (g.w[:, None] * np.abs(t)).sum()
    for p in range(3):
        m = g.part == p
        assert np.abs((g.w[m, None] * t[m]).sum(0)).max() < 1e-12 * scale
        assert abs((g.w[m] * (o.e3[m] * t[m]).sum(1)).sum()) < 1e-12 * scale


def test_traction_brute_force_on_an_ellipse():
    A, B, phi, c = 1.3, 0.6, -0.4, np.array([0.0, 0.5])
    p = np.array([[ELLIPSE, c[0], c[1], phi, A, B]])
    o = so.StokesOracle(p, 16, 16)
    g = o.geom
    sig = np.array([_density(t) for t in g.t]).ravel()
    t_h = ((o.operators[0] - 0.5 * np.eye(2 * o.n)) @ sig).reshape(-1, 2)
    pos, der = _ellipse_curve(A, B, phi, c)
    for i in (3, 100, 200):
        ti = g.t[i]
        ref = np.zeros(2)
        for comp in range(2):
            def f(s):
                if s == ti:
                    return 0.0
                return (so.traction_kernel(g.x[i] - pos(s), g.nu[i]) @ _density(s))[comp] * \
                    np.linalg.norm(der(s))
            ref[comp] = sum(si.quad(f, a, b, limit=400, epsabs=1e-15, epsrel=1e-14)[0]
                            for a, b in ((ti - math.pi, ti), (ti, ti + math.pi)))
        assert np.abs(t_h[i] - ref).max() < 1e-12, (i, t_h[i] - ref)


# --------------------------------------------------------------------------
# mobility
# --------------------------------------------------------------------------

@pytest.mark.parametrize("a,mu", [(1.0, 1.0), (1.5, 0.7)])
def test_single_disk_mobility(a, mu):
    """Torque: rotlet, omega = tau / (4 pi mu a^2), v = 0. Force: the disk
    moves with the single layer of a uniform density, v = F (1 - 2 log a) /
    (8 pi mu) (the log's reference length is the unit of length)."""
    o = so.StokesOracle(_disk(a), 16, 16, mu)
    r = o.mobility([0.0, 0.0], [1.3])
    assert abs(r["omega"][0] - 1.3 / (4 * math.pi * mu * a * a)) < 1e-14
    assert np.abs(r["v"]).max() < 1e-15
    F = np.array([0.7, -0.2])
    r = o.mobility(F, [0.0])
    assert np.abs(r["v"][0] - F * (1 - 2 * math.log(a)) / (8 * math.pi * mu)).max() < 1e-14
    assert abs(r["omega"][0]) < 1e-15


def _mobility_matrix(o):
    n = len(o.particles)
    M = np.zeros((3 * n, 3 * n))
    for k in range(3 * n):
        e = np.zeros(3 * n)
        e[k] = 1.0
        r = o.mobility(e[:2 * n].reshape(n, 2), e[2 * n:])
        M[:, k] = np.concatenate([r["v"].ravel(), r["omega"]])
    return M


def test_mobility_rigid_motion_loads_and_reciprocity():
    p = _three()
    o = so.StokesOracle(p, 16, 16, 1.2)
    g = o.geom
    rng = np.random.default_rng(4)
    F = rng.standard_normal((3, 2))
    tau = rng.standard_normal(3)
    r = o.mobility(F, tau)
    # u on each boundary is the rigid motion v + omega (x - a)^perp
    rig = r["v"][g.part] + r["omega"][g.part, None] * o.e3
    assert np.abs(r["u"] - rig).max() < 1e-10 * np.abs(r["u"]).max()
    # sigma carries exactly the given force and torque, mu none
    s = r["sigma"].reshape(-1, 2)
    Fs = np.stack([np.bincount(g.part, g.w * s[:, 0]), np.bincount(g.part, g.w * s[:, 1])], -1)
    assert np.abs(Fs - F).max() < 1e-12
    assert np.abs(np.bincount(g.part, g.w * (o.e3 * s).sum(1)) - tau).max() < 1e-12
    # Lorentz reciprocity: symmetric mobility matrix
    M = _mobility_matrix(o)
    assert np.abs(M - M.T).max() < 1e-10 * np.abs(M).max()
    # loads free of net force and torque (about the origin) dissipate
    n = len(p)
    C = np.zeros((3, 3 * n))
    for i in range(n):
        C[0, 2 * i] = C[1, 2 * i + 1] = 1.0
        C[2, 2 * n + i] = 1.0
        C[2, 2 * i] = -p[i, 2]
        C[2, 2 * i + 1] = p[i, 1]
    _, _, Vt = np.linalg.svd(C)
    Z = Vt[3:].T
    ev = np.linalg.eigvalsh(Z.T @ (0.5 * (M + M.T)) @ Z)
    assert ev.min() > 0, ev


def test_mobility_converges_under_refinement():
    p = _three()
    F = np.array([[0.3, -0.1], [0.2, 0.5], [-0.5, -0.4]])
    tau = np.array([0.2, -0.7, 0.4])
    r16 = so.StokesOracle(p, 16, 16).mobility(F, tau)
    r24 = so.StokesOracle(p, 24, 16).mobility(F, tau)
    assert np.abs(r16["v"] - r24["v"]).max() < 1e-10
    assert np.abs(r16["omega"] - r24["omega"]).max() < 1e-10


def test_two_distant_disks_point_force_limit():
    """Disks at distance d under F and -F: each moves with its own single-
    disk velocity plus the stokeslet flow of the other, up to O(1/d^2)."""
    d = 40.0
    p = np.array([[DISK, 0.0, 0.0, 0.0, 1.0, 1.0], [DISK, d * 0.6, d * 0.8, 1.0, 1.0, 1.0]])
    F = np.array([0.4, 0.9])
    r = so.StokesOracle(p, 16, 16).mobility(np.stack([F, -F]), [0.0, 0.0])
    G = so.stokeslet(p[0, 1:3] - p[1, 1:3])
    v1 = F / (8 * math.pi) - G @ F
    assert np.abs(r["v"][0] - v1).max() < 2.0 / d ** 2
    assert np.abs(r["v"][1] + v1).max() < 2.0 / d ** 2


def test_mobility_step_is_forward_euler():
    o = so.StokesOracle(_disk(1.0, 0.0, 0.0, 0.25), 16, 16)
    r = o.mobility([0.0, 0.0], [2.0])
    q = so.mobility_step(o.particles, r["v"], r["omega"], 0.05)
    assert abs(q[0, 3] - (0.25 + 0.05 * 2.0 / (4 * math.pi))) < 1e-15
    assert np.abs(q[0, 1:3]).max() < 1e-15


# --------------------------------------------------------------------------
# the pins catch planted mistakes
# --------------------------------------------------------------------------

def _pins_ok():
    try:
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            test_single_layer_on_a_circle(2.5, 2.0)
            test_traction_identities()
            test_single_disk_mobility(1.5, 0.7)
            p = _three()[:2]
            o = so.StokesOracle(p, 12, 16)
            r = o.mobility([[0.3, -0.2], [0.1, 0.4]], [0.5, -0.3])
            g = o.geom
            rig = r["v"][g.part] + r["omega"][g.part, None] * o.e3
            assert np.abs(r["u"] - rig).max() < 1e-10 * np.abs(r["u"]).max()
    except (AssertionError, np.linalg.LinAlgError):
        return False
    return True


def test_planted_mistakes_are_caught(monkeypatch):
    assert _pins_ok()
    orig_tk, orig_curv = so.traction_kernel, so.curvature
    orig_blocks, orig_inc = so.single_layer_blocks, so.StokesOracle.incident_density
    orig_avg = so.StokesOracle.rigid_average
    M = so.log_moments(16)
    mistakes = [
        ("traction sign", so, "traction_kernel", lambda r, n: -orig_tk(r, n)),
        ("tangent for the normal", so, "traction_kernel",
         lambda r, n: orig_tk(r, np.stack([n[..., 1], -n[..., 0]], -1))),
        ("diagonal limit dropped", so, "curvature", lambda *a: 0.0 * orig_curv(*a)),
        ("log sign", so, "single_layer_blocks",
         lambda lw, w, rr, mu: orig_blocks(-lw, w, rr, mu)),
        ("dyad dropped", so, "single_layer_blocks",
         lambda lw, w, rr, mu: orig_blocks(lw, w, 0 * rr, mu)),
        ("neighbour moments swapped", so, "log_moments", lambda n: M[[0, 2, 1]]),
        ("torque normaliser", so.StokesOracle, "incident_density",
         lambda self, F, tau: orig_inc(self, F, np.asarray(tau) * 0.5)),
        ("angular velocity sign", so.StokesOracle, "rigid_average",
         lambda self, u: (orig_avg(self, u)[0], -orig_avg(self, u)[1])),
    ]
    for name, target, attr, value in mistakes:
        with monkeypatch.context() as m:
            m.setattr(target, attr, value)
            assert not _pins_ok(), name
