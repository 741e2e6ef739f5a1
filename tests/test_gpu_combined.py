"""The combined representation u = D[sigma] + eta S[sigma] on the GPU
(YK_REP_COMBINED; the remark on Eq. bwform, real coupling), against the
FP64 oracle with the same eta, through the C ABI:
  * the operator 1/2 I + D + eta S (FP64): 1e-12 relative, like the double
    layer's FP64 operator, with the dense and the cut-off far field;
  * its normal derivative (exterior limit): 1e-11 relative;
  * solve, forces and torques at the default tolerance: 1e-9;
  * the off-surface field: 1e-12;
  * particles in near contact (oversampled quadrature of both kernels);
  * at rho = 16 plain GMRES needs fewer iterations than for the double layer;
  * the combinations it does not support are refused.
"""
import numpy as np
import pytest

from oracle import yk_oracle as yo
from paper_1810_04131_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ETA = 0.25


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
    return yk.params_for(wl, precision=yk.YK_FP64, representation=yk.YK_REP_COMBINED,
                         bw_eta=ETA, **kw)


@pytest.mark.parametrize("rho", [4.0, 8.0])
def test_combined_operator_solve_forces(yk, ctx, rho):
    wl = W.small_system(3, 81, shape=W.SHAPE_ELLIPSE, n_panels=12, rho=rho, A=1.0, B=0.5, gap=0.3)
    o = yo.Oracle(wl.particles, wl.n_panels, wl.n_gl, rho, yo.QBXParams(order=wl.qbx_order), eta=ETA)
    A, Gn = o.dense(want_grad=True)
    rng = np.random.default_rng(int(rho))
    sig = rng.standard_normal(A.shape[0])
    for ff in (yk.YK_FARFIELD_DENSE, yk.YK_FARFIELD_CUTOFF):
        g = yk.Geometry(ctx, wl.particles, _params(yk, wl, farfield=ff))
        assert rel(g.yk_matvec(sig, yk.YK_FP64), A @ sig) < 1e-12
        un = g.yk_normal_derivative(sig, yk.YK_FP64)
        ref = Gn @ sig
        assert np.abs(un - ref).max() <= 1e-12 * (np.abs(Gn) @ np.abs(sig)).max() + \
            1e-11 * np.abs(ref).max()
        g.close()
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl))
    f = g.yk_label(yk.YK_LABEL_TANH, 10.0)
    s, F, tau, info = g.yk_solve_forces(f)
    s_ref = np.linalg.solve(A, f)
    F_ref, tau_ref, _ = o.forces_torques(f, Gn @ s_ref)
    assert info["rel_residual"] <= 1e-12
    assert rel(s, s_ref) < 1e-9
    scale = np.abs(F_ref).max()
    assert np.abs(F.reshape(-1, 2) - F_ref).max() < 1e-9 * scale
    assert np.abs(tau - tau_ref).max() < 1e-9 * max(scale, np.abs(tau_ref).max())
    T = W.off_surface_targets(wl.particles, 40, wl.box, 0.5, seed=5)
    assert rel(g.yk_eval_potential(s, T), o.potential(s_ref, T)) < 1e-11
    g.close()


def test_combined_near_contact(yk, ctx):
    """Two disks 0.05 apart: the other disk's near panels are integrated on
    their oversampled nodes for both kernels of the combined operator."""
    parts = np.array([[0, 0.0, 0.0, 0.2, 1.0, 1.0], [0, 2.05, 0.3, 1.0, 1.0, 1.0]])
    wl = W.Workload("contact", parts, rho=4.0, n_panels=16, n_gl=16, qbx_order=10)
    o = yo.Oracle(parts, 16, 16, 4.0, yo.QBXParams(order=10), eta=ETA)
    assert o.contact_panels(0) or o.contact_panels(300)
    A, Gn = o.dense(want_grad=True)
    sig = np.random.default_rng(3).standard_normal(A.shape[0])
    g = yk.Geometry(ctx, parts, _params(yk, wl))
    assert rel(g.yk_matvec(sig, yk.YK_FP64), A @ sig) < 1e-12
    un = g.yk_normal_derivative(sig, yk.YK_FP64)
    assert np.abs(un - Gn @ sig).max() <= 1e-11 * (np.abs(Gn) @ np.abs(sig)).max()
    g.close()


def test_combined_helps_plain_gmres_at_large_rho(yk, ctx):
    wl = W.small_system(6, 13, shape=W.SHAPE_ELLIPSE, n_panels=16, rho=16.0, A=1.0, B=0.5, gap=0.3)
    its = {}
    for rep in (yk.YK_REP_DOUBLE_LAYER, yk.YK_REP_COMBINED):
        g = yk.Geometry(ctx, wl.particles, yk.params_for(
            wl, precision=yk.YK_FP64, representation=rep, bw_eta=ETA, precond=yk.YK_PRECOND_NONE))
        _, info = g.yk_solve(g.yk_label(yk.YK_LABEL_TANH, 10.0))
        assert info["converged"]
        its[rep] = info["iterations"]
        g.close()
    assert its[yk.YK_REP_COMBINED] < 0.75 * its[yk.YK_REP_DOUBLE_LAYER], its


def test_combined_refuses_unsupported(yk, ctx):
    wl = W.small_system(2, 82, n_panels=8, rho=4.0)
    for kw in (dict(precision=yk.YK_MIXED), dict(bw_eta=0.0), dict(bw_eta=-1.0)):
        prm = yk.params_for(wl, representation=yk.YK_REP_COMBINED,
                            **{**dict(precision=yk.YK_FP64, bw_eta=ETA), **kw})
        with pytest.raises(yk.YKError) as e:
            yk.Geometry(ctx, wl.particles, prm)
        assert e.value.code == yk.YK_ERR_ARG
    g = yk.Geometry(ctx, wl.particles, _params(yk, wl))
    with pytest.raises(yk.YKError) as e:
        g.yk_eval_potential_near(np.zeros(g.n), np.array([[10.0, 10.0]]))
    assert e.value.code == yk.YK_ERR_ARG
    g.close()
