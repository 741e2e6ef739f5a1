"""The Stokes mobility step on the GPU (yk_stokes_apply, yk_mobility, yk_step
with mobility = 1; Section 3, Eqs. stokes, mobility_bc, stokesjump,
mobilityu, mob_vec) against the FP64 oracle (oracle/stokes_oracle.py),
through the C ABI:
  * the three boundary operators (interior traction 1/2 I + K*, the completed
    operator with the rigid-motion projector W, the on-surface single layer
    S) on disks and turned ellipses, for two panel layouts, close particles
    (node-by-node sums) and spread ones (particle expansions for far pairs):
    1e-12 relative in FP64, 1e-6 with the FP32 far field;
  * v, omega and the density of the mobility problem, FP64 and mixed
    precision, at the default tolerance: 1e-10 (close particles, spread ones,
    and 30 disks at Table 2's density and 10 x 7 nodes);
  * a single disk under a torque turns at tau / (4 pi mu a^2);
  * one step of Algorithm 1 with the mobility velocities against the oracle's
    Yukawa solve, forces, repulsion, mobility and Euler update;
  * at 64 particles (no dense oracle): the boundary velocity is rigid, the
    density carries the loads, FP64 and mixed agree;
  * arguments it does not support are refused.
"""
import math

import numpy as np
import pytest

from oracle import stokes_oracle as so
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


def _three():
    return np.array([[W.SHAPE_DISK, 0.0, 0.0, 0.3, 1.0, 1.0],
                     [W.SHAPE_ELLIPSE, 2.6, 0.4, 1.1, 1.0, 0.5],
                     [W.SHAPE_DISK, 0.5, 2.5, 2.0, 0.8, 0.8]])


def _geom(yk, ctx, parts, npan=16, ngl=16, **kw):
    wl = W.Workload("stokes", parts, rho=1.0, n_panels=npan, n_gl=ngl, qbx_order=10)
    return yk.Geometry(ctx, parts, yk.params_for(wl, **kw))


def _spread():
    """12 ellipses over a 31 x 31 box: most particle pairs are far (centre
    distance >= 2 (r_P + r_Q)) and go through the particle expansions."""
    return W.small_system(12, 41, shape=W.SHAPE_ELLIPSE, n_panels=12, A=1.0, B=0.5,
                          gap=0.3).particles


@pytest.mark.parametrize("case,npan,ngl", [("three", 16, 16), ("three", 12, 10),
                                           ("spread", 12, 16)])
def test_stokes_operators_match_oracle(yk, ctx, case, npan, ngl):
    parts = _three() if case == "three" else _spread()
    o = so.StokesOracle(parts, npan, ngl, viscosity=1.3)
    A0, A, S = o.operators
    g = _geom(yk, ctx, parts, npan, ngl, viscosity=1.3)
    sig = np.random.default_rng(npan).standard_normal(2 * o.n)
    for op, M in ((yk.YK_STOKES_TRACTION, A0), (yk.YK_STOKES_COMPLETED, A),
                  (yk.YK_STOKES_VELOCITY, S)):
        got = g.yk_stokes_apply(sig, op, yk.YK_FP64)
        assert rel(got, M @ sig) < 1e-12, (op, rel(got, M @ sig))
    got = g.yk_stokes_apply(sig, yk.YK_STOKES_COMPLETED, yk.YK_MIXED)
    assert rel(got, A @ sig) < 1e-6
    g.close()


def _table2_like():
    """30 unit disks at Table 2's density and discretisation (10 panels x 7
    nodes, gap >= 0.5): near and far pairs, 70 nodes per particle."""
    return W.small_system(30, 43, n_panels=10, n_gl=7, rho=4.0, gap=0.5).particles


@pytest.mark.parametrize("case,precision", [("three", "fp64"), ("three", "mixed"),
                                            ("spread", "fp64"), ("spread", "mixed"),
                                            ("table2", "fp64"), ("table2", "mixed")])
def test_mobility_matches_oracle(yk, ctx, case, precision):
    parts = {"three": _three, "spread": _spread, "table2": _table2_like}[case]()
    npan, ngl = {"three": (16, 16), "spread": (12, 16), "table2": (10, 7)}[case]
    rng = np.random.default_rng(7)
    F = rng.standard_normal((len(parts), 2))
    tau = rng.standard_normal(len(parts))
    o = so.StokesOracle(parts, npan, ngl, viscosity=0.8)
    ref = o.mobility(F, tau)
    prec = yk.YK_FP64 if precision == "fp64" else yk.YK_MIXED
    g = _geom(yk, ctx, parts, npan, ngl, precision=prec, viscosity=0.8)
    v, om, sig, info = g.yk_mobility(F, tau, want_sigma=True)
    assert info["rel_residual"] <= 1e-12, info
    assert (info["refinements"] > 0) == (precision == "mixed")
    assert rel(sig, ref["sigma"]) < 1e-10
    scale = max(np.abs(ref["v"]).max(), np.abs(ref["omega"]).max())
    assert np.abs(v - ref["v"]).max() < 1e-10 * scale
    assert np.abs(om - ref["omega"]).max() < 1e-10 * scale
    g.close()


def test_single_disk_turns_as_a_rotlet(yk, ctx):
    a, mu, tq = 1.5, 0.7, 1.3
    g = _geom(yk, ctx, np.array([[W.SHAPE_DISK, 3.0, -1.0, 0.4, a, a]]), viscosity=mu,
              precision=yk.YK_FP64)
    v, om, _, _ = g.yk_mobility([[0.0, 0.0]], [tq])
    assert abs(om[0] - tq / (4 * math.pi * mu * a * a)) < 1e-13
    assert np.abs(v).max() < 1e-14
    g.close()


def test_mobility_step_matches_oracle(yk, ctx):
    """Algorithm 1 with the Stokes mobility: yk_step(mobility=1) against the
    oracle's dense Yukawa solve, forces and torques, repulsion, mobility
    solve of the total loads and forward Euler (Eq. mob_vec)."""
    parts = W.make_particles(3, 7.0, 0.3, seed=11, shape=W.SHAPE_ELLIPSE, A=1.0, B=0.5)
    wl = W.Workload("mob3", parts, rho=1.0, n_panels=16, n_gl=16, qbx_order=10)
    g = yk.Geometry(ctx, parts, yk.params_for(wl))
    dyn = dict(dt=0.5, c0=0.01, q=3, label_kind=1, label_param=2.0, mobility=1)
    d = yk.default_dynamics(**dyn)
    ref = parts.copy()
    for _ in range(2):
        got, _, _ = g.yk_step(1, **dyn)
        o = yo.Oracle(ref, 16, 16, 1.0, yo.QBXParams(order=10))
        res = yo.solve_dense(o, yo.label(o.geom, 1, 2.0))
        Fr, taur, _ = yo.repulsion(ref, d.c0, d.q)
        m = so.StokesOracle(ref, 16, 16).mobility(res["F"] + Fr, res["tau"] + taur)
        ref = so.mobility_step(ref, m["v"], m["omega"], d.dt)
        assert np.abs(got[:, 1:4] - ref[:, 1:4]).max() < 1e-10
    assert np.abs(ref[:, 1:4] - parts[:, 1:4]).max() > 1e-4     # the particles moved
    g.close()


def test_mobility_64_particles_properties(yk, ctx):
    """64 disks and ellipses (16,384 nodes): S[sigma] moves every boundary
    rigidly with the returned (v, omega), sigma carries the loads, and the
    FP64 and mixed solves agree."""
    wl = W.small_system(64, 31, shape=W.SHAPE_ELLIPSE, n_panels=16, rho=1.0, A=1.0, B=0.5,
                        gap=0.3)
    rng = np.random.default_rng(8)
    F = rng.standard_normal((64, 2))
    F -= F.mean(0)
    tau = rng.standard_normal(64)
    out = {}
    for prec in (yk.YK_FP64, yk.YK_MIXED):
        g = yk.Geometry(ctx, wl.particles, yk.params_for(wl, precision=prec))
        v, om, sig, info = g.yk_mobility(F, tau, want_sigma=True)
        assert info["rel_residual"] <= 1e-12
        out[prec] = (v, om, sig)
        if prec == yk.YK_FP64:
            xy, nrm, w = g.yk_nodes()
            u = g.yk_stokes_apply(sig, yk.YK_STOKES_VELOCITY).reshape(-1, 2)
            part = np.repeat(np.arange(64), g.n // 64)
            d = xy - wl.particles[part, 1:3]
            rig = v[part] + om[part, None] * np.stack([-d[:, 1], d[:, 0]], -1)
            assert np.abs(u - rig).max() < 1e-9 * np.abs(u).max()
            s = sig.reshape(-1, 2)
            Fs = np.stack([np.bincount(part, w * s[:, 0]), np.bincount(part, w * s[:, 1])], -1)
            assert np.abs(Fs - F).max() < 1e-11
            ts = np.bincount(part, w * (d[:, 0] * s[:, 1] - d[:, 1] * s[:, 0]))
            assert np.abs(ts - tau).max() < 1e-11
        g.close()
    a, b = out[yk.YK_FP64], out[yk.YK_MIXED]
    assert rel(b[2], a[2]) < 1e-10
    assert np.abs(b[0] - a[0]).max() < 1e-10 * np.abs(a[0]).max()
    assert np.abs(b[1] - a[1]).max() < 1e-10 * np.abs(a[1]).max()


def test_stokes_refuses_unsupported(yk, ctx):
    g = _geom(yk, ctx, _three()[:1], npan=2, ngl=16)
    with pytest.raises(yk.YKError) as e:
        g.yk_mobility([[0.0, 0.0]], [1.0])
    assert e.value.code == yk.YK_ERR_ARG
    g.close()
    g = _geom(yk, ctx, _three()[:1])
    with pytest.raises(yk.YKError) as e:
        g.yk_stokes_apply(np.zeros(2 * g.n), 7)
    assert e.value.code == yk.YK_ERR_ARG
    with pytest.raises(yk.YKError) as e:
        g.yk_step(1, mobility=2)
    assert e.value.code == yk.YK_ERR_ARG
    g.close()
    wl = W.Workload("s", _three()[:1], rho=1.0, n_panels=16, n_gl=16, qbx_order=10)
    with pytest.raises(yk.YKError) as e:
        yk.Geometry(ctx, wl.particles, yk.params_for(wl, viscosity=0.0))
    assert e.value.code == yk.YK_ERR_ARG
