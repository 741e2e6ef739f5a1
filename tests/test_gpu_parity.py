"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (relative 2-norm unless stated):
  * FP64 matvec: 1e-12;
  * mixed (FP32 far field) matvec: 1e-6;
  * density after a solve at the library's default tolerance (residual
    1e-12; forces amplify the density error about 25x at rho = 4, which is
    why the default is not 1e-10), and forces/torques (max-norm relative to
    max |F|): 1e-9;
  * normal derivative: its rows cancel (entries ~10x the result), so the
    difference is bounded by 1e-12 |G| |sigma| and 1e-11 relative;
  * the FP32 far field of one distant source disk, row by row: 1e-6 +
    3e-7 z'_max of the sum of absolute pair contributions (the FP32 error
    of the exponent grows with the scaled distance z').
Small systems span several 256-target tiles with a ragged tail; the
512-disk system is checked on sampled rows and through properties that
hold at any size (the oracle's residual of the GPU density).
"""
import numpy as np
import pytest

from oracle import yk_oracle as yo
from paper_1810_04131_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def yk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_04131_gb300 import yk as Y
    Y.load()
    return Y


@pytest.fixture(scope="module")
def ctx(yk):
    c = yk.Context(0)
    yield c
    c.close()


def _params(yk, wl, **kw):
    return yk.params_for(wl, **kw)


SMALL = {
    # name: (workload builder, extra oracle/gpu params)
    "disks5_pan9": lambda: W.small_system(5, 21, n_panels=9, n_gl=16, rho=0.7, qbx_order=10),
    "ellipses4_gl11": lambda: W.small_system(4, 22, shape=W.SHAPE_ELLIPSE, n_panels=12, n_gl=11,
                                             rho=1.3, qbx_order=9, A=1.0, B=0.5, gap=0.3),
    "disks2_allnear": lambda: W.small_system(2, 23, n_panels=3, n_gl=16, rho=0.5, qbx_order=8),
    # 320 nodes per particle: several 256-node chunks per particle pair
    "disks3_npp320": lambda: W.small_system(3, 24, n_panels=20, n_gl=16, rho=0.6, qbx_order=10),
    "single_disk": lambda: W.Workload("single", np.array([[0, 0.3, -0.2, 0.4, 1.0, 1.0]]),
                                      rho=4.0, n_panels=16, n_gl=16, qbx_order=10),
}


@pytest.fixture(scope="module")
def dense_cache():
    return {}


def _oracle(wl, dense_cache, want_grad=True):
    key = wl.name
    if key not in dense_cache:
        o = yo.Oracle(wl.particles, wl.n_panels, wl.n_gl, wl.rho, yo.QBXParams(order=wl.qbx_order))
        A, Gn = o.dense(want_grad=True)
        dense_cache[key] = (o, A, Gn)
    return dense_cache[key]


@pytest.mark.parametrize("name", list(SMALL))
def test_geometry_and_label(yk, ctx, name):
    wl = SMALL[name]()
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl))
    o = yo.make_geometry(wl.particles, wl.n_panels, wl.n_gl)
    xy, nrm, w = g.yk_nodes()
    assert np.abs(xy - o.x).max() < 1e-13
    assert np.abs(nrm - o.nu).max() < 1e-14
    assert np.abs(w - o.w).max() < 1e-15
    for kind, par in ((0, 10.0), (1, 2.0), (1, 6.0), (2, 0.0)):
        assert np.abs(g.yk_label(kind, par) - yo.label(o, kind, par)).max() < 1e-14


@pytest.mark.parametrize("name", list(SMALL))
def test_matvec_and_gradient_small(yk, ctx, dense_cache, name):
    wl = SMALL[name]()
    o, A, Gn = _oracle(wl, dense_cache)
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl))
    rng = np.random.default_rng(5)
    for sig in (rng.standard_normal(g.n), yo.label(o.geom, 0, 10.0)):
        y64 = g.yk_matvec(sig, yk.YK_FP64)
        assert rel(y64, A @ sig) < 1e-12
        y32 = g.yk_matvec(sig, yk.YK_MIXED)
        assert rel(y32, A @ sig) < 1e-6
        # the normal-derivative rows have entries ~10x the result (they
        # cancel), so bound the difference by the rows' magnitude
        cond = np.abs(Gn) @ np.abs(sig)
        un64 = g.yk_normal_derivative(sig, yk.YK_FP64)
        assert np.abs(un64 - Gn @ sig).max() < 1e-12 * cond.max()
        assert rel(un64, Gn @ sig) < 1e-11
        unsp = g.yk_normal_derivative(sig, yk.YK_MIXED)
        assert np.abs(unsp - Gn @ sig).max() < 1e-12 * cond.max()
        assert rel(unsp, Gn @ sig) < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["disks5_pan9", "ellipses4_gl11"])
def test_solve_forces_small(yk, ctx, dense_cache, name, precision):
    wl = SMALL[name]()
    o, A, Gn = _oracle(wl, dense_cache)
    prec = yk.YK_FP64 if precision == "fp64" else yk.YK_MIXED
    # a 1e-12 residual keeps the solver's own error well inside the 1e-9 bar
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl, precision=prec))
    f = g.yk_label(0, 10.0)
    sig, info = g.yk_solve(f)
    s_ref = np.linalg.solve(A, f)
    assert info["converged"] and info["rel_residual"] <= 1e-12
    assert rel(sig, s_ref) < 1e-9
    F, tau, net = g.yk_forces_torques(sig, f)
    F_ref, tau_ref, tau0_ref = o.forces_torques(f, Gn @ s_ref)
    scale = np.abs(F_ref).max()
    assert np.abs(F - F_ref).max() < 1e-9 * scale
    assert np.abs(tau - tau_ref).max() < 1e-9 * max(scale, np.abs(tau_ref).max())
    assert np.abs(net[:2] - F_ref.sum(0)).max() < 1e-9 * scale


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["disks5_pan9", "ellipses4_gl11"])
def test_energy_small(yk, ctx, dense_cache, name, precision):
    """Energy of Eq. main (boundary form) from the same density: per-particle
    parts and total against the oracle's, to the normal derivative's bar."""
    wl = SMALL[name]()
    o, A, Gn = _oracle(wl, dense_cache)
    prec = yk.YK_FP64 if precision == "fp64" else yk.YK_MIXED
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl, precision=prec))
    f = g.yk_label(1, 2.0)
    s = np.linalg.solve(A, f)
    phi, total = g.yk_energy(s, f)
    ref = o.energy(f, Gn @ s)
    scale = np.abs(o.geom.w * f).sum() * (np.abs(Gn) @ np.abs(s)).max() * wl.rho
    assert np.abs(phi - ref).max() < 1e-12 * scale
    assert abs(total - ref.sum()) < 1e-12 * scale


def test_forces_are_minus_energy_gradient_gpu(yk, ctx):
    """Section 7.1 on the GPU path: centered differences (eps = 1e-3) of the
    energy after moving or turning one particle (yk_update_geometry, mixed
    solves to 1e-12) against yk_forces_torques, as in the oracle's pin."""
    parts = W.make_particles(3, 7.0, 0.3, seed=11, shape=W.SHAPE_ELLIPSE, A=1.0, B=0.5)
    wl = W.Workload("fd3", parts, rho=1.0, n_panels=16, n_gl=16, qbx_order=10)
    g = yk.Geometry(ctx, parts, _params(yk, wl))

    def solve(P):
        g.yk_update_geometry(P)
        f = g.yk_label(1, 2.0)
        s, info = g.yk_solve(f)
        assert info["converged"]
        return f, s

    f0, s0 = solve(parts)
    F0, tau0, _ = g.yk_forces_torques(s0, f0)
    F0 = F0.reshape(-1, 2)
    eps = 1e-3
    Ffd, tfd = np.zeros((3, 2)), np.zeros(3)
    for i in range(3):
        for k, col in enumerate((1, 2, 3)):
            E = []
            for sgn in (1.0, -1.0):
                P = parts.copy()
                P[i, col] += sgn * eps
                f, s = solve(P)
                E.append(g.yk_energy(s, f)[1])
            d = -(E[0] - E[1]) / (2 * eps)
            if k < 2:
                Ffd[i, k] = d
            else:
                tfd[i] = d
    sc = np.abs(F0).max()
    assert sc > 0.1
    assert np.abs(Ffd - F0).max() < 2e-5 * sc
    assert np.abs(tfd - tau0).max() < 2e-5 * sc


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_block_preconditioner(yk, ctx, dense_cache, precision):
    """Right preconditioning by the inverse self-interaction block of each
    particle changes the iteration count, not the solution."""
    wl = SMALL["ellipses4_gl11"]()
    o, A, Gn = _oracle(wl, dense_cache)
    prec = yk.YK_FP64 if precision == "fp64" else yk.YK_MIXED
    s_ref = None
    its = {}
    for pc in (yk.YK_PRECOND_NONE, yk.YK_PRECOND_BLOCK):
        g = yk.Geometry(ctx, wl.particles, _params(yk, wl, precision=prec, precond=pc))
        f = g.yk_label(0, 10.0)
        s, info = g.yk_solve(f)
        s_ref = np.linalg.solve(A, f) if s_ref is None else s_ref
        assert info["converged"] and rel(s, s_ref) < 1e-9
        its[pc] = info["iterations"]
        g.close()
    assert its[yk.YK_PRECOND_BLOCK] < its[yk.YK_PRECOND_NONE]


def test_disks8_end_to_end(yk, ctx, dense_cache):
    """8 disks, N = 2048, rho = 1, QBX order 8, tol 1e-10: density,
    potential at 1000 off-surface targets, forces and torques, both modes."""
    wl = W.disks8()
    o, A, Gn = _oracle(wl, dense_cache)
    f_ref = yo.label(o.geom, 0, 10.0)
    s_ref = np.linalg.solve(A, f_ref)
    F_ref, tau_ref, _ = o.forces_torques(f_ref, Gn @ s_ref)
    u_ref = o.potential(s_ref, wl.targets)
    for prec in (yk.YK_FP64, yk.YK_MIXED):
        g = yk.Geometry(ctx, wl.particles, _params(yk, wl, precision=prec))
        f = g.yk_label(0, 10.0)
        assert np.abs(f - f_ref).max() < 1e-13
        sig, info = g.yk_solve(f)
        assert info["converged"]
        assert rel(sig, s_ref) < 1e-9
        F, tau, net = g.yk_forces_torques(sig, f)
        sc = np.abs(F_ref).max()
        assert np.abs(F - F_ref).max() < 1e-9 * sc
        assert np.abs(tau - tau_ref).max() < 1e-9 * sc
        u = g.yk_eval_potential(sig, wl.targets)
        assert rel(u, u_ref) < 1e-9
        g.close()


def test_cutoff_far_field(yk, ctx, dense_cache):
    """Cut-off far field: a source particle is dropped when its whole
    contribution is bounded below cutoff_tol * max|sigma|. On a sparse
    system (many pairs beyond the cut-off) the FP64 cut-off operator stays
    within a few cutoff_tol of the dense one, and a mixed cut-off solve
    matches the oracle's dense solution."""
    wl = W.small_system(24, 31, n_panels=8, n_gl=16, rho=0.5, qbx_order=10, gap=0.4)
    wl.particles[:, 1:3] *= 2.5   # spread out: box ~ 2.5x larger
    o = yo.Oracle(wl.particles, wl.n_panels, wl.n_gl, wl.rho, yo.QBXParams(order=wl.qbx_order))
    A, Gn = o.dense(want_grad=True)
    rng = np.random.default_rng(9)
    sig = rng.standard_normal(A.shape[0])
    for tol in (1e-8, 1e-15):
        g = yk.Geometry(ctx, wl.particles, _params(yk, wl, farfield=yk.YK_FARFIELD_CUTOFF,
                                                   cutoff_tol=tol))
        y = g.yk_matvec(sig, yk.YK_FP64)
        assert np.abs(y - A @ sig).max() <= 20 * tol * np.abs(sig).max() + 1e-13
        y32 = g.yk_matvec(sig, yk.YK_MIXED)
        assert rel(y32, A @ sig) < 1e-6
        # normal derivative: FP64 tiles, expansions and FP32 far pairs all in play
        cond = (np.abs(Gn) @ np.abs(sig)).max()   # the gradient rows cancel (see above)
        for prec in (yk.YK_FP64, yk.YK_MIXED):
            un = g.yk_normal_derivative(sig, prec)
            assert np.abs(un - Gn @ sig).max() <= 1e-12 * cond + 40 * tol * np.abs(sig).max() / wl.rho
        g.close()
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl, farfield=yk.YK_FARFIELD_CUTOFF,
                                               precision=yk.YK_MIXED))
    f = g.yk_label(0, 10.0)
    s, info = g.yk_solve(f)
    assert info["converged"] and rel(s, np.linalg.solve(A, f)) < 1e-9
    # the cut-off drops something here (otherwise the test would be vacuous)
    gd = yk.Geometry(ctx, wl.particles, _params(yk, wl, farfield=yk.YK_FARFIELD_CUTOFF,
                                                cutoff_tol=1e-3))
    assert rel(gd.yk_matvec(sig, yk.YK_FP64), A @ sig) > 1e-8


def test_fmm_far_field_against_direct_sums(yk, ctx):
    """FMM far field (expansions in FP64): with the density nonzero on one
    particle only, a target more than three leaf sides away from it (in x or
    y) has no source in its near list, so it receives the expansions' value
    alone. That value is checked against the direct double-layer sum with the
    oracle's kernel at orders 12 and 20 (sources and targets spread over
    every level of the tree: rho = 2 reaches across the whole box)."""
    wl = W.small_system(60, 41, n_panels=8, n_gl=16, rho=2.0, qbx_order=10, gap=0.4)
    geo = yo.make_geometry(wl.particles, wl.n_panels, wl.n_gl)
    npp = wl.n_panels * wl.n_gl
    rng = np.random.default_rng(17)
    leaf = 8.0
    c = wl.particles[:, 1:3]
    for P in (7, 33):
        sl = slice(P * npp, (P + 1) * npp)
        sig = np.zeros(geo.w.size)
        sig[sl] = 1.0 + 0.3 * np.cos(3 * geo.t[sl]) + 0.2 * rng.standard_normal(npp)
        ws = geo.w[sl] * sig[sl]
        far = np.maximum(np.abs(c[:, 0] - c[P, 0]), np.abs(c[:, 1] - c[P, 1])) > 3 * leaf
        rows = np.flatnonzero(np.repeat(far, npp))
        assert rows.size > 1000
        ref = np.array([(yo.dl_kernel(geo.x[r][None], geo.x[sl], geo.nu[sl], wl.rho) * ws).sum()
                        for r in rows])
        assert np.abs(ref).max() > 1e-8 * np.abs(ws).sum()   # not negligible
        errs = {}
        for order, tol in ((12, 1e-8), (20, 1e-11)):
            g = yk.Geometry(ctx, wl.particles, _params(yk, wl, farfield=yk.YK_FARFIELD_FMM,
                                                       fmm_order=order, fmm_leaf=leaf))
            y = g.yk_matvec(sig, yk.YK_MIXED)
            errs[order] = np.abs(y[rows] - ref).max()
            assert errs[order] <= tol * np.abs(ws).sum(), (P, order, errs[order])
            g.close()
        assert errs[20] < errs[12]


def test_fmm_operator_and_solve(yk, ctx):
    """YK_FARFIELD_FMM as the inner operator of the mixed solver: the FP32
    operator (FP32 near lists + FMM far field) within the FP32 bar of the
    dense operator, for a given and an autotuned leaf size; the FP64 path and
    the refinement residual use the cut-off operator, so a mixed FMM solve
    matches the oracle's dense solution and forces to 1e-9."""
    wl = W.small_system(24, 31, n_panels=8, n_gl=16, rho=1.5, qbx_order=10, gap=0.4)
    wl.particles[:, 1:3] *= 2.5
    o = yo.Oracle(wl.particles, wl.n_panels, wl.n_gl, wl.rho, yo.QBXParams(order=wl.qbx_order))
    A, Gn = o.dense(want_grad=True)
    rng = np.random.default_rng(19)
    sig = rng.standard_normal(A.shape[0])
    for leaf in (6.0, 0.0):
        g = yk.Geometry(ctx, wl.particles, _params(yk, wl, farfield=yk.YK_FARFIELD_FMM,
                                                   fmm_leaf=leaf))
        y32 = g.yk_matvec(sig, yk.YK_MIXED)
        assert rel(y32, A @ sig) < 1e-6
        # repeatable up to the order of the near field's FP64 atomic adds
        # (the symmetric kernel over the near lists' particle pairs)
        assert rel(g.yk_matvec(sig, yk.YK_MIXED), y32) < 1e-15
        y64 = g.yk_matvec(sig, yk.YK_FP64)
        assert np.abs(y64 - A @ sig).max() <= 20 * 1e-15 * np.abs(sig).max() + 1e-13
        g.close()
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl, farfield=yk.YK_FARFIELD_FMM, fmm_leaf=6.0,
                                               precision=yk.YK_MIXED))
    f = g.yk_label(0, 10.0)
    s, info = g.yk_solve(f)
    s_ref = np.linalg.solve(A, f)
    assert info["converged"] and rel(s, s_ref) < 1e-9
    F, tau, net = g.yk_forces_torques(s, f)
    F_ref, tau_ref, _ = o.forces_torques(f, Gn @ s_ref)
    scale = np.abs(F_ref).max()
    assert np.abs(F - F_ref).max() < 1e-9 * scale
    assert np.abs(tau - tau_ref).max() < 1e-9 * max(scale, np.abs(tau_ref).max())
    # moving the particles rebuilds the tree: the moved system still matches
    moved = wl.particles.copy()
    moved[:, 1] += 0.37
    moved[:, 3] += 0.2
    g.yk_update_geometry(moved)
    o2 = yo.Oracle(moved, wl.n_panels, wl.n_gl, wl.rho, yo.QBXParams(order=wl.qbx_order))
    rows = np.sort(rng.choice(A.shape[0], 40, replace=False))
    y32 = g.yk_matvec(sig, yk.YK_MIXED)
    ref = o2.apply_rows(sig, rows)
    assert np.abs(y32[rows] - ref).max() < 1e-6 * np.abs(A @ sig).max()


def test_fmm_without_admissible_leaf_falls_back_to_cutoff(yk, ctx):
    """When no leaf size satisfies the FMM's accuracy conditions (here order 4
    at rho = 0.5: a leaf would have to be both wider than 2.9 radii and
    narrower than 0.7), the inner operator's far field is the cut-off P2P."""
    wl = W.small_system(24, 31, n_panels=8, n_gl=16, rho=0.5, qbx_order=10, gap=0.4)
    rng = np.random.default_rng(20)
    sig = rng.standard_normal(24 * 128)
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl, farfield=yk.YK_FARFIELD_FMM, fmm_order=4))
    gc = yk.Geometry(ctx, wl.particles, _params(yk, wl, farfield=yk.YK_FARFIELD_CUTOFF))
    # the same operator, up to the order of the symmetric kernel's FP64 atomic adds
    y, yc = g.yk_matvec(sig, yk.YK_MIXED), gc.yk_matvec(sig, yk.YK_MIXED)
    assert rel(y, yc) < 1e-15


def test_repulsion_matches_oracle(yk, ctx):
    """Eq. repul with the circle decomposition of Section S1 (ellipses and
    disks together): force, torque and potential against the oracle."""
    p = np.array([[1, 0.0, 0.0, 0.3, 1.0, 0.5], [0, 2.5, 0.4, 0.0, 1.0, 1.0],
                  [1, 0.5, 2.2, 1.2, 1.0, 0.5], [0, -2.4, 1.1, 0.5, 1.0, 1.0]])
    wl = W.Workload("rep4", p, rho=1.0, n_panels=8, n_gl=16)
    g = yk.Geometry(ctx, p, _params(yk, wl))
    F, tau, phi = g.yk_repulsion(0.01, 3)
    Fr, taur, phir = yo.repulsion(p, 0.01, 3)
    sc = np.abs(Fr).max()
    assert np.abs(F - Fr).max() < 1e-14 * sc
    assert np.abs(tau - taur).max() < 1e-14 * sc
    assert np.abs(phi - phir).max() < 1e-14 * np.abs(phir).max()


def test_dynamics_steps_match_oracle(yk, ctx):
    """Algorithm 1 with constant drag (Eq. euler): three steps of yk_step on
    three close ellipses (mixed solves to 1e-12, warm-started) against the
    oracle's exact discrete solve, forces, repulsion and Euler update; the
    step energies (Eq. main plus the repulsion potential) as well."""
    parts = W.make_particles(3, 7.0, 0.3, seed=11, shape=W.SHAPE_ELLIPSE, A=1.0, B=0.5)
    wl = W.Workload("dyn3", parts, rho=1.0, n_panels=16, n_gl=16, qbx_order=10)
    g = yk.Geometry(ctx, parts, _params(yk, wl))
    dyn = dict(dt=0.5, c0=0.01, q=3, label_kind=1, label_param=2.0)
    d = yk.default_dynamics(**dyn)
    ref = parts.copy()
    for step in range(3):
        got, energy, info = g.yk_step(1, **dyn)
        o = yo.Oracle(ref, 16, 16, 1.0, yo.QBXParams(order=10))
        f = yo.label(o.geom, 1, 2.0)
        res = yo.solve_dense(o, f)
        Fr, taur, phir = yo.repulsion(ref, d.c0, d.q)
        e_ref = o.energy(f, res["un"]).sum() + phir.sum()
        assert abs(energy[0] - e_ref) < 1e-10 * abs(e_ref)
        ref = yo.euler_step(ref, res["F"] + Fr, res["tau"] + taur, d.dt, d.xi_x, d.xi_theta)
        assert np.abs(got[:, 1:4] - ref[:, 1:4]).max() < 1e-10
    assert np.abs(ref[:, 1:4] - parts[:, 1:4]).max() > 1e-3       # the particles moved


def test_dynamics_warm_start_saves_iterations(yk, ctx):
    """The previous step's density as the initial guess (Algorithm 1 marching
    in time) needs fewer GMRES iterations than a cold start, and ends at the
    same configuration to the solve tolerance."""
    wl = W.small_system(24, 61, n_panels=12, n_gl=16, rho=1.0, qbx_order=10, gap=0.4)
    runs = {}
    for warm in (1, 0):
        g = yk.Geometry(ctx, wl.particles, _params(yk, wl))
        parts, energy, infos = g.yk_step(5, dt=0.05, warm_start=warm)
        runs[warm] = (parts, [i["iterations"] for i in infos])
        g.close()
    assert sum(runs[1][1][1:]) < sum(runs[0][1][1:])
    assert np.abs(runs[1][0][:, 1:4] - runs[0][0][:, 1:4]).max() < 1e-8


def _near_targets_disk():
    xs = np.linspace(-2.5, 2.5, 200)
    X, Y = np.meshgrid(xs, xs)
    T = np.stack([X.ravel(), Y.ravel()], 1)
    T = T[np.hypot(T[:, 0], T[:, 1]) > 1.0][::7]
    ang = np.linspace(0, 2 * np.pi, 49)[:-1] + 0.013
    rings = [np.stack([(1 + d) * np.cos(ang), (1 + d) * np.sin(ang)], 1)
             for d in (1e-9, 1e-6, 1e-3, 0.02, 0.05, 0.1, 0.2, 0.4)]
    return np.concatenate([T] + rings + [np.array([[0.3, -0.2]])])   # last one inside


def test_potential_near_boundary_single_disk(yk, ctx):
    """yk_eval_potential_near (QBX next to the boundary) on Table 1's grid
    and on rings 1e-9 to 0.4 off a rotated disk (rho = 4): against the
    oracle's near evaluation of the same density and against Eq. true_soln;
    NaN inside the particle."""
    parts = np.array([[0, 0.0, 0.0, 0.4, 1.0, 1.0]])
    wl = W.Workload("disk_near", parts, rho=4.0, n_panels=16, n_gl=16, qbx_order=10)
    o = yo.Oracle(parts, 16, 16, 4.0, yo.QBXParams(order=10))
    s = np.linalg.solve(o.dense(), yo.label(o.geom, 2))
    g = yk.Geometry(ctx, parts, _params(yk, wl))
    T = _near_targets_disk()
    u = g.yk_eval_potential_near(s, T)
    assert np.isnan(u[-1]) and np.isfinite(u[:-1]).all()
    ref = o.potential_near(s, T[:-1])
    assert np.abs(u[:-1] - ref).max() < 1e-12
    c, s_ = np.cos(0.4), np.sin(0.4)
    Tb = np.stack([c * T[:-1, 0] + s_ * T[:-1, 1], -s_ * T[:-1, 0] + c * T[:-1, 1]], 1)
    import scipy.special as sp
    r = np.hypot(Tb[:, 0], Tb[:, 1])
    ue = 0.5 * (sp.k0(r / 4.0) / sp.k0(0.25) + sp.k1(r / 4.0) / sp.k1(0.25) * Tb[:, 0] / r)  # Eq. true_soln
    assert np.abs(u[:-1] - ue).max() < 1e-10


def test_potential_near_boundary_close_ellipses(yk, ctx):
    """Three close ellipses (one target can be near two of them): the GPU
    near evaluation against the oracle's on targets 1e-8 to 0.3 off the
    boundaries along the normals, and against the far-field path where the
    targets are far from every boundary."""
    parts = W.make_particles(3, 7.0, 0.3, seed=11, shape=W.SHAPE_ELLIPSE, A=1.0, B=0.5)
    wl = W.Workload("ell_near", parts, rho=1.0, n_panels=16, n_gl=16, qbx_order=10)
    o = yo.Oracle(parts, 16, 16, 1.0, yo.QBXParams(order=10))
    f = yo.label(o.geom, 0, 10.0)
    s = np.linalg.solve(o.dense(), f)
    rng = np.random.default_rng(23)
    T = []
    for prt in parts:
        for tt in rng.uniform(0, 2 * np.pi, 10):
            x, dx = yo.curve(prt, np.array([tt]))
            nu = np.array([dx[0, 1], -dx[0, 0]]) / np.hypot(*dx[0])
            for d in (1e-8, 1e-4, 0.01, 0.05, 0.15, 0.3):
                T.append(x[0] + d * nu)
    T = np.array(T)
    inside = np.zeros(len(T), bool)
    for prt in parts:
        c, s_ = np.cos(prt[3]), np.sin(prt[3])
        dv = T - prt[1:3]
        lx, ly = c * dv[:, 0] + s_ * dv[:, 1], -s_ * dv[:, 0] + c * dv[:, 1]
        inside |= (lx / prt[4]) ** 2 + (ly / prt[5]) ** 2 < 1.0
    g = yk.Geometry(ctx, parts, _params(yk, wl))
    u = g.yk_eval_potential_near(s, T)
    assert (np.isnan(u) == inside).all()
    ref = o.potential_near(s, T[~inside])
    assert np.abs(u[~inside] - ref).max() < 1e-12 * np.abs(ref).max()
    xs = np.linspace(-4.0, 11.0, 16)
    X, Y = np.meshgrid(xs, xs)
    far = np.stack([X.ravel(), Y.ravel()], 1)
    dmin = np.min(np.hypot(far[:, None, 0] - parts[None, :, 1], far[:, None, 1] - parts[None, :, 2]), 1)
    far = far[dmin > 2.5]
    uf = g.yk_eval_potential(s, far)
    assert np.abs(g.yk_eval_potential_near(s, far) - uf).max() < 1e-14 * np.abs(uf).max()


def test_forces_are_not_pairwise(yk, ctx):
    """Section 'Pairwise potentials': the force on each particle of a
    six-particle cluster, F_i (all particles in the fluid), against the sum
    of its two-particle forces f_i = sum_j f_ij (only P_i and P_j in the
    fluid). Every f_ij matches the oracle's exact two-particle solve (to 1e-9
    of the cluster's largest force); F_i and f_i differ by well over the
    solver tolerance, as the paper reports."""
    parts = W.make_particles(6, 9.0, 0.3, seed=31, shape=W.SHAPE_ELLIPSE, A=1.0, B=0.5)
    wl = W.Workload("pair6", parts, rho=1.0, n_panels=16, n_gl=16, qbx_order=10)
    g = yk.Geometry(ctx, parts, _params(yk, wl))
    f = g.yk_label(0, 10.0)
    sig, F, tau, info = g.yk_solve_forces(f)
    F = F.reshape(-1, 2)
    fp = np.zeros_like(F)
    for i in range(6):
        for j in range(i + 1, 6):
            pair = parts[[i, j]]
            g2 = yk.Geometry(ctx, pair, _params(yk, wl))
            f2 = g2.yk_label(0, 10.0)
            _, F2, _, _ = g2.yk_solve_forces(f2)
            F2 = F2.reshape(-1, 2)
            o = yo.Oracle(pair, 16, 16, 1.0, yo.QBXParams(order=10))
            r = yo.solve_dense(o, yo.label(o.geom, 0, 10.0))
            # a far pair's net force is small (its stress integrand cancels), so
            # the bar is relative to the cluster's force scale
            assert np.abs(F2 - r["F"]).max() < 1e-9 * np.abs(F).max()
            fp[i] += F2[0]
            fp[j] += F2[1]
            g2.close()
    rel = np.hypot(*(F - fp).T) / np.hypot(*F.T)
    assert rel.max() > 1e-2             # not pairwise additive
    assert np.isfinite(rel).all()


@pytest.mark.parametrize("shape,gap", [(W.SHAPE_DISK, 0.05), (W.SHAPE_ELLIPSE, 0.02)])
def test_near_contact_matches_oracle(yk, ctx, shape, gap):
    """Particles closer than the configurations' gaps: another particle's
    panels next to a target are integrated on their oversampled nodes, in
    every operator. FP64 and mixed operators and their normal derivatives
    against the oracle's (same rule), and a mixed solve with forces."""
    A, B = (1.0, 1.0) if shape == W.SHAPE_DISK else (1.0, 0.5)
    parts = np.array([[shape, 0.0, 0.0, 0.3 * (shape == 0), A, B],
                      [shape, 2.0 + gap, 0.0, 1.1 * (shape == 0), A, B],
                      [shape, 0.7, 3.1, 0.5, A, B]])
    wl = W.Workload("contact", parts, rho=1.0, n_panels=16, n_gl=16, qbx_order=10)
    o = yo.Oracle(parts, 16, 16, 1.0, yo.QBXParams(order=10))
    A_, Gn = o.dense(want_grad=True)
    assert sum(len(o.contact_panels(i)) for i in range(o.geom.n)) > 0     # the rule is in play
    rng = np.random.default_rng(29)
    sig = rng.standard_normal(A_.shape[0])
    cond = (np.abs(Gn) @ np.abs(sig)).max()
    for prec in ("fp64", "mixed"):
        p_ = yk.YK_FP64 if prec == "fp64" else yk.YK_MIXED
        g = yk.Geometry(ctx, parts, _params(yk, wl, precision=p_))
        y64 = g.yk_matvec(sig, yk.YK_FP64)
        assert rel(y64, A_ @ sig) < 1e-12
        assert rel(g.yk_matvec(sig, yk.YK_MIXED), A_ @ sig) < 1e-6
        un = g.yk_normal_derivative(sig, p_)
        assert np.abs(un - Gn @ sig).max() < 1e-12 * cond
        f = g.yk_label(0, 10.0)
        s, info = g.yk_solve(f)
        s_ref = np.linalg.solve(A_, f)
        assert info["converged"] and rel(s, s_ref) < 1e-9
        F, tau, _ = g.yk_forces_torques(s, f)
        F_ref, tau_ref, _ = o.forces_torques(f, Gn @ s_ref)
        sc = np.abs(F_ref).max()
        assert np.abs(F.reshape(-1, 2) - F_ref).max() < 1e-9 * sc
        assert np.abs(tau - tau_ref).max() < 1e-9 * max(sc, np.abs(tau_ref).max())
        g.close()


def test_device_pointers_match_host(yk, ctx):
    import torch
    wl = SMALL["disks5_pan9"]()
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl))
    rng = np.random.default_rng(3)
    sig = rng.standard_normal(g.n)
    y_h = g.yk_matvec(sig, yk.YK_FP64)
    sd = torch.from_numpy(sig).cuda()
    yd = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    g.yk_matvec(sd, yk.YK_FP64, out=yd)
    torch.cuda.synchronize()
    # the FP64 tiles accumulate with atomics, so the summation order varies
    assert rel(yd.cpu().numpy(), y_h) < 1e-15


def test_errors_and_edge_cases(yk, ctx):
    wl = SMALL["disks5_pan9"]()
    # overlapping particles
    bad = np.array([[0, 0.0, 0.0, 0.0, 1.0, 1.0], [0, 0.5, 0.0, 0.0, 1.0, 1.0]])
    with pytest.raises(yk.YKError) as e:
        yk.Geometry(ctx, bad, _params(yk, wl))
    assert e.value.code == yk.YK_ERR_BAD_GEOMETRY
    # parameters out of range
    for kw in (dict(n_gl=1), dict(n_gl=40), dict(qbx_order=30), dict(rho=-1.0),
               dict(oversample=0), dict(near_width=-1), dict(precision=7), dict(farfield=3),
               dict(fmm_order=1), dict(fmm_order=31), dict(fmm_leaf=-1.0)):
        with pytest.raises(yk.YKError) as e:
            yk.Geometry(ctx, wl.particles, _params(yk, wl, **kw))
        assert e.value.code == yk.YK_ERR_ARG
    # not converged: outputs still written, residual reported
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl, precision=yk.YK_FP64, max_iter=2))
    f = g.yk_label(0, 10.0)
    sig, info = g.yk_solve(f, allow_not_converged=True)
    assert not info["converged"] and info["iterations"] == 2
    assert np.isfinite(sig).all() and 0 < info["rel_residual"] < 1
    # zero data -> zero density
    z, info = g.yk_solve(np.zeros(g.n))
    assert np.all(z == 0)
    # warm start from the exact solution converges at once
    g2 = yk.Geometry(ctx, wl.particles, _params(yk, wl, precision=yk.YK_FP64))
    s, _ = g2.yk_solve(f)
    s2, info2 = g2.yk_solve(f, sigma0=s)
    assert info2["iterations"] <= 1 and rel(s2, s) < 1e-10
    # empty target list
    assert g2.yk_eval_potential(s, np.zeros((0, 2))).size == 0


def test_allocation_failure_is_an_error_not_a_fault(yk, ctx):
    """Fault injection on the host side: a geometry whose Krylov basis cannot
    fit in device memory (1001 x 2^28 doubles, ~2 TB) fails with
    YK_ERR_NO_MEMORY, frees what it took, and the context keeps working."""
    n_particles = (1 << 28) // 256
    parts = np.zeros((n_particles, 6))
    parts[:, 0] = 0
    parts[:, 1] = (np.arange(n_particles) % 4096) * 3.0
    parts[:, 2] = (np.arange(n_particles) // 4096) * 3.0
    parts[:, 4] = parts[:, 5] = 1.0
    wl = SMALL["disks5_pan9"]()
    with pytest.raises(yk.YKError) as e:
        yk.Geometry(ctx, parts, _params(yk, wl, n_panels=16, n_gl=16, gmres_restart=1000,
                                        precond=yk.YK_PRECOND_NONE))
    assert e.value.code == yk.YK_ERR_NO_MEMORY
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl))
    assert np.isfinite(g.yk_matvec(np.ones(g.n), yk.YK_FP64)).all()
    g.close()


def test_serving_failed_request_does_not_stop_others(yk):
    """A corrupted request (overlapping particles) fails with
    YK_ERR_BAD_GEOMETRY; requests around it complete."""
    ctx = yk.Context(0)
    good = W.small_system(3, 50, n_panels=8)
    bad = np.array([[0, 0.0, 0.0, 0.0, 1.0, 1.0], [0, 0.5, 0.0, 0.0, 1.0, 1.0]])
    ids = [ctx.yk_submit(good.particles, _params(yk, good)),
           ctx.yk_submit(bad, _params(yk, good)),
           ctx.yk_submit(good.particles, _params(yk, good))]
    with pytest.raises(yk.YKError):
        ctx.yk_drain()
    r0 = ctx.yk_poll(ids[0], n_nodes=good.n_nodes, n_particles=3)
    assert r0["status"] == yk.YK_REQ_DONE
    with pytest.raises(yk.YKError) as e:
        ctx.yk_poll(ids[1])
    assert e.value.code == yk.YK_ERR_BAD_GEOMETRY
    r2 = ctx.yk_poll(ids[2], n_nodes=good.n_nodes, n_particles=3)
    assert r2["status"] == yk.YK_REQ_DONE
    assert rel(r2["sigma"], r0["sigma"]) < 1e-12
    ctx.close()


def test_serving_alone_and_in_mix(yk):
    """Continuous batching: requests of different sizes, shapes and rho,
    submitted together (several in flight at once on different streams),
    give the same density, forces and torques as each solved alone."""
    ctx = yk.Context(0)
    # (particles, panels, rho, shape, far field); the FMM requests tune their
    # leaf size when solved alone and reuse the cached choice in the mix
    dense, fmm = yk.YK_FARFIELD_DENSE, yk.YK_FARFIELD_FMM
    specs = [(3, 8, 0.5, 0, dense), (6, 10, 1.0, 1, dense), (2, 16, 2.0, 0, dense),
             (9, 8, 1.0, 1, dense), (14, 12, 0.5, 0, dense), (5, 20, 2.0, 1, dense),
             (1, 16, 1.0, 0, dense), (11, 9, 1.0, 0, dense), (7, 14, 0.5, 1, dense),
             (4, 24, 2.0, 0, dense), (16, 8, 1.0, 1, dense), (8, 11, 2.0, 0, dense),
             (40, 8, 1.0, 0, fmm), (30, 10, 2.0, 1, fmm)]
    wls, prms = [], []
    for k, (n, npan, rho, shape, ff) in enumerate(specs):
        wls.append(W.small_system(n, 40 + k, shape=shape, n_panels=npan, rho=rho,
                                  A=1.0, B=0.5 if shape else 1.0, gap=0.3))
        prms.append(_params(yk, wls[-1], farfield=ff))
    alone = []
    for wl, prm in zip(wls, prms):
        g = yk.Geometry(ctx, wl.particles, prm)
        f = g.yk_label(0, 10.0)
        s, F, tau, info = g.yk_solve_forces(f)
        alone.append((s, F.reshape(-1), tau))
        g.close()
    ids = [ctx.yk_submit(wl.particles, prm) for wl, prm in zip(wls, prms)]
    # poll while requests are in flight, then drain the rest
    seen = {}
    for _ in range(3):
        for wl, rid in zip(wls, ids):
            if rid in seen:
                continue
            r = ctx.yk_poll(rid, n_nodes=wl.n_nodes, n_particles=wl.n_particles)
            assert r["status"] in (yk.YK_REQ_QUEUED, yk.YK_REQ_RUNNING, yk.YK_REQ_DONE)
            if r["status"] == yk.YK_REQ_DONE:
                seen[rid] = r
    ctx.yk_drain()
    # the force unit of these systems (gamma = 1, unit particles): the largest
    # force over the set. An isolated particle feels no net force (the energy
    # of Eq. main does not change when it translates), so its own max|F| is
    # discretisation noise and no scale for a relative bound.
    fscale = max(np.abs(a[1]).max() for a in alone)
    for wl, rid, (s, F, tau) in zip(wls, ids, alone):
        r = seen.get(rid) or ctx.yk_poll(rid, n_nodes=wl.n_nodes, n_particles=wl.n_particles)
        assert r["status"] == yk.YK_REQ_DONE
        assert rel(r["sigma"], s) < 1e-11
        sc = max(np.abs(F).max(), fscale)
        assert np.abs(r["F"] - F).max() < 1e-9 * sc
        assert np.abs(r["tau"] - tau).max() < 1e-9 * max(sc, np.abs(tau).max())
        assert r["latency_ms"] > 0
        with pytest.raises(yk.YKError):   # collected requests are released
            ctx.yk_poll(rid)
    ctx.close()


# --------------------------------------------------------------------------
# FP32 far field, one source particle at a time: every evaluation mode of
# the FP32 kernels (close pairs, the full and the short K1 fit, the narrow
# expansions of degree 4 and 3, the exact-zero skip) against the oracle.
# The density is zero on the target disk, so its rows hold the far field of
# the source disk alone, which in a full system would be hidden under the
# near field by many orders of magnitude. Each pair carries an FP32 error
# of about 2e-7 z' relative (the rounding of the scaled positions and of
# 1/z' enters the exponent), so the bound is taken against the sum of the
# absolute pair contributions, |A| |sigma|, which a random density makes
# far larger than the cancelling sum itself.
# --------------------------------------------------------------------------

LOG2E = 1.4426950408889634


@pytest.mark.parametrize("rho,D,mode", [
    (1.0, 3.0, "close"), (1.0, 8.0, "full fit"), (1.0, 20.0, "short fit"),
    (1.0, 40.0, "narrow"), (1.0, 80.0, "narrow3"), (1.0, 95.0, "zero"),
    (4.0, 30.0, "full fit"), (4.0, 50.0, "narrow"), (4.0, 80.0, "narrow3"),
    (0.25, 12.0, "short fit"), (0.25, 30.0, "zero")])
def test_far_field_modes_one_source(yk, ctx, rho, D, mode):
    a = 0.7
    parts = np.array([[0, 0.0, 0.0, 0.3, 1.0, 1.0],
                      [0, D * np.cos(a), D * np.sin(a), 1.1, 1.0, 1.0]])
    wl = W.Workload("two_disks", parts, rho=rho, n_panels=16, n_gl=16, qbx_order=10)
    g = yk.Geometry(ctx, parts, _params(yk, wl))
    o = yo.Oracle(parts, 16, 16, rho, yo.QBXParams(order=10))
    A = o.dense()
    rng = np.random.default_rng(int(D * 10 + rho * 100))
    sig = np.zeros(g.n)
    sig[256:] = rng.standard_normal(256)
    rows = np.arange(256)
    y32 = g.yk_matvec(sig, yk.YK_MIXED)[rows]
    y64 = g.yk_matvec(sig, yk.YK_FP64)[rows]
    ref = A[rows] @ sig
    absum = np.abs(A[rows]) @ np.abs(sig)
    assert np.all(np.abs(y64 - ref) <= 1e-13 * absum)
    gap = D - 2.0
    if mode == "zero":
        # every pair's exp2(-z') flushes to zero in FP32: exactly nothing
        assert gap * LOG2E / rho >= 128
        assert np.all(y32 == 0.0)
        assert absum.max() < 1e-37
        return
    zmax = (D + 2.0) * LOG2E / rho
    tol = 1e-6 + 3e-7 * zmax
    err = np.abs(y32 - ref) / absum
    assert err.max() <= tol, (mode, err.max(), tol)


# --------------------------------------------------------------------------
# full size (512 disks, N = 131072): sampled rows and properties
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big(yk, ctx):
    wl = W.disks512()
    o = yo.Oracle(wl.particles, wl.n_panels, wl.n_gl, wl.rho, yo.QBXParams(order=wl.qbx_order))
    return wl, o


def test_full_size_matvec_sampled(yk, ctx, big):
    wl, o = big
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl))
    rng = np.random.default_rng(11)
    sig = rng.standard_normal(g.n)
    rows = np.sort(rng.choice(g.n, 48, replace=False))
    ref = o.apply_rows(sig, rows)
    y64 = g.yk_matvec(sig, yk.YK_FP64)
    assert rel(y64[rows], ref) < 1e-12
    y32 = g.yk_matvec(sig, yk.YK_MIXED)
    assert rel(y32[rows], ref) < 1e-6
    # whole-vector agreement of the two precisions (any size)
    assert rel(y32, y64) < 1e-6
    # the precision-split normal derivative against the FP64 one (any size)
    u64 = g.yk_normal_derivative(sig, yk.YK_FP64)
    usp = g.yk_normal_derivative(sig, yk.YK_MIXED)
    assert rel(usp, u64) < 1e-11


def test_full_size_mixed_solve_properties(yk, ctx, big):
    """Mixed solve on the 512-disk system: the oracle's residual of the GPU
    density at sampled rows, and forces of sampled particles recomputed by
    the oracle from the GPU density."""
    wl, o = big
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl, precision=yk.YK_MIXED))
    f = g.yk_label(0, 10.0)
    sig, info = g.yk_solve(f)
    assert info["converged"] and info["rel_residual"] <= 1e-10
    rng = np.random.default_rng(12)
    rows = np.sort(rng.choice(g.n, 48, replace=False))
    res = f[rows] - o.apply_rows(sig, rows)
    assert np.abs(res).max() < 1e-9 * np.abs(f).max()
    F, tau, net = g.yk_forces_torques(sig, f)
    for p in rng.choice(wl.n_particles, 2, replace=False):
        idx = np.arange(p * 256, (p + 1) * 256)
        _, un = o.apply_rows(sig, idx, want_grad=True)
        full = np.zeros(g.n)
        full[idx] = un
        F_o, tau_o, _ = o.forces_torques(f, full)
        sc = np.abs(F).max()   # the error measure is relative to max_i |F_i|
        assert np.abs(F[p] - F_o[p]).max() < 1e-9 * sc
        assert abs(tau[p] - tau_o[p]) < 1e-9 * sc
