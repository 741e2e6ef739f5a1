"""Coarse-space deflation of the inner GMRES (YK_COARSE_MODES, the default of
the mixed solve) through the C ABI:
  * the deflated solve reaches the FP64 oracle's dense solution of Eq. bie
    (disks and ellipses, rho = 1 and 4) at the library's default tolerance;
  * on 64-particle systems it gives the same density as block Jacobi alone
    and takes fewer inner (FP32) GMRES iterations;
  * it is not used where it does not apply: FP64 precision, one particle,
    near-contact panels (the iteration counts equal those without it).
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


def _solve(yk, ctx, wl, **kw):
    g = yk.Geometry(ctx, wl.particles, yk.params_for(wl, **kw))
    f = g.yk_label(0, 10.0)
    sig, info = g.yk_solve(f)
    g.close()
    return f, sig, info


@pytest.mark.parametrize("shape,rho", [(W.SHAPE_DISK, 1.0), (W.SHAPE_DISK, 4.0),
                                       (W.SHAPE_ELLIPSE, 1.0), (W.SHAPE_ELLIPSE, 4.0)])
def test_coarse_solve_matches_oracle(yk, ctx, shape, rho):
    wl = W.small_system(6, 17, shape=shape, n_panels=16, rho=rho, A=1.0,
                        B=0.5 if shape == W.SHAPE_ELLIPSE else 1.0, gap=0.4)
    f, sig, info = _solve(yk, ctx, wl, coarse=yk.YK_COARSE_MODES)
    assert info["converged"] and info["rel_residual"] <= 1e-12
    assert info["coarse_dim"] == 3 * len(wl.particles)
    o = yo.Oracle(wl.particles, wl.n_panels, wl.n_gl, rho, yo.QBXParams(order=wl.qbx_order))
    ref = np.linalg.solve(o.dense(), f)
    assert rel(sig, ref) < 1e-9


@pytest.mark.parametrize("shape,rho", [(W.SHAPE_DISK, 1.0), (W.SHAPE_DISK, 4.0),
                                       (W.SHAPE_ELLIPSE, 1.0)])
def test_coarse_takes_fewer_inner_iterations(yk, ctx, shape, rho):
    wl = W.small_system(64, 23, shape=shape, n_panels=16, rho=rho, A=1.0,
                        B=0.5 if shape == W.SHAPE_ELLIPSE else 1.0, gap=0.3)
    _, s0, i0 = _solve(yk, ctx, wl, coarse=yk.YK_COARSE_NONE)
    _, s1, i1 = _solve(yk, ctx, wl, coarse=yk.YK_COARSE_MODES)
    assert i0["converged"] and i1["converged"]
    assert i0["rel_residual"] <= 1e-12 and i1["rel_residual"] <= 1e-12
    assert rel(s1, s0) < 1e-10
    assert i0["coarse_dim"] == 0 and i1["coarse_dim"] == 3 * 64
    print("inner iterations without / with the coarse space:", i0["iterations"],
          i1["iterations"], "refinements", i0["refinements"], i1["refinements"])
    assert i1["iterations"] < i0["iterations"]


def test_coarse_not_used_where_it_does_not_apply(yk, ctx):
    wl = W.small_system(12, 29, n_panels=16, gap=0.3)
    _, s1, i1 = _solve(yk, ctx, wl)
    assert i1["coarse_dim"] == 36                       # the default for the mixed solve
    _, s0, i0 = _solve(yk, ctx, wl, precision=yk.YK_FP64)
    assert i0["converged"] and i0["coarse_dim"] == 0    # FP64 precision
    one = W.Workload("one", wl.particles[:1], rho=1.0, n_panels=16, n_gl=16, qbx_order=10)
    _, _, i2 = _solve(yk, ctx, one)
    assert i2["converged"] and i2["coarse_dim"] == 0    # one particle
    _, _, i3 = _solve(yk, ctx, wl, precond=yk.YK_PRECOND_NONE)
    assert i3["converged"] and i3["coarse_dim"] == 0    # no block preconditioner
    # two disks 0.07 apart: near-contact panels
    p = np.array([[W.SHAPE_DISK, 0.0, 0.0, 0.0, 1.0, 1.0],
                  [W.SHAPE_DISK, 2.05, 0.3, 0.0, 1.0, 1.0],
                  [W.SHAPE_DISK, -1.0, 4.0, 0.0, 1.0, 1.0]])
    near = W.Workload("contact", p, rho=1.0, n_panels=16, n_gl=16, qbx_order=10)
    f, s4, i4 = _solve(yk, ctx, near)
    assert i4["converged"] and i4["coarse_dim"] == 0
    o = yo.Oracle(p, 16, 16, 1.0, yo.QBXParams(order=10))
    # the oracle's near-contact rows (Green's identity pins them) against the dense solve
    assert rel(s4, np.linalg.solve(o.dense(), f)) < 1e-9


def test_coarse_refused_values(yk, ctx):
    wl = W.small_system(2, 3, n_panels=8)
    with pytest.raises(yk.YKError) as e:
        yk.Geometry(ctx, wl.particles, yk.params_for(wl, coarse=2))
    assert e.value.code == yk.YK_ERR_ARG
