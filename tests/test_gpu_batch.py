"""Batched solves (yk_solve_batch): several independent configurations of
Eq. (bie) whose inner FP32 GMRES advance in lock step, one launch per stage
for all of them.

Checked through the C ABI:
  * each system's density equals that of its own yk_solve within 1e-10
    relative (both solve to the default residual 1e-12, so the two differ
    only by where each refinement stopped);
  * the batch includes systems that cannot take the batched path (FP64, FMM
    far field), which are solved one by one with the same result;
  * one batched system against the FP64 oracle's dense solution and forces
    (1e-9, the bar for density and forces);
  * host and device arrays both work; a geometry given twice, or geometries of
    two contexts, are refused.
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


SPECS = [  # (particles, panels, rho, shape, precision, far field)
    (3, 8, 0.5, 0, "mixed", "dense"), (6, 10, 1.0, 1, "mixed", "dense"),
    (2, 16, 2.0, 0, "mixed", "dense"), (9, 8, 1.0, 1, "mixed", "dense"),
    (14, 12, 0.5, 0, "mixed", "dense"), (1, 16, 1.0, 0, "mixed", "dense"),
    (11, 9, 1.0, 0, "fp64", "dense"), (24, 8, 1.5, 0, "mixed", "fmm"),
    (5, 20, 2.0, 1, "mixed", "dense"), (7, 14, 0.5, 1, "mixed", "dense"),
]


def _systems(yk, ctx):
    out = []
    for k, (n, npan, rho, shape, prec, ff) in enumerate(SPECS):
        wl = W.small_system(n, 60 + k, shape=shape, n_panels=npan, rho=rho, A=1.0,
                            B=0.5 if shape else 1.0, gap=0.3)
        if ff == "fmm":
            wl.particles[:, 1:3] *= 2.5
        prm = yk.params_for(wl, precision=yk.YK_MIXED if prec == "mixed" else yk.YK_FP64,
                            farfield=yk.YK_FARFIELD_FMM if ff == "fmm" else yk.YK_FARFIELD_DENSE)
        out.append((wl, yk.Geometry(ctx, wl.particles, prm)))
    return out


def test_batch_matches_separate_solves(yk):
    import torch
    ctx = yk.Context(0, torch.cuda.current_stream().cuda_stream)
    try:
        systems = _systems(yk, ctx)
        fs = [g.yk_label(yk.YK_LABEL_TANH, 10.0) for _, g in systems]
        alone = [g.yk_solve(f)[0] for (_, g), f in zip(systems, fs)]
        sig, infos = yk.yk_solve_batch([g for _, g in systems], fs)
        for k, (s, s0, info) in enumerate(zip(sig, alone, infos)):
            assert info["rel_residual"] <= 1e-12, (k, info)
            assert info["iterations"] > 0, (k, info)
            # refinement steps only in mixed precision
            assert (info["refinements"] > 0) == (SPECS[k][4] == "mixed"), (k, info)
            assert rel(s, s0) < 1e-10, (k, rel(s, s0))
        # device arrays, second call on the same geometries (workspaces reused)
        dev = torch.device("cuda", 0)
        fd = [torch.from_numpy(f).to(dev) for f in fs]
        sd = [torch.zeros(g.n, dtype=torch.float64, device=dev) for _, g in systems]
        yk.yk_solve_batch([g for _, g in systems], fd, sd)
        for s, s0 in zip(sd, alone):
            assert rel(s.cpu().numpy(), s0) < 1e-10
    finally:
        ctx.close()


def test_batch_against_oracle(yk):
    import torch
    ctx = yk.Context(0, torch.cuda.current_stream().cuda_stream)
    try:
        wls = [W.small_system(4, 71, shape=1, n_panels=10, rho=1.3, A=1.0, B=0.5, gap=0.3),
               W.small_system(3, 72, n_panels=9, rho=0.7)]
        gs = [yk.Geometry(ctx, wl.particles, yk.params_for(wl, precision=yk.YK_MIXED)) for wl in wls]
        fs = [g.yk_label(yk.YK_LABEL_TANH, 10.0) for g in gs]
        sig, _ = yk.yk_solve_batch(gs, fs)
        for wl, g, f, s in zip(wls, gs, fs, sig):
            o = yo.Oracle(wl.particles, wl.n_panels, wl.n_gl, wl.rho,
                          yo.QBXParams(order=wl.qbx_order))
            A, Gn = o.dense(want_grad=True)
            s_ref = np.linalg.solve(A, f)
            assert rel(s, s_ref) < 1e-9
            F, tau, _ = g.yk_forces_torques(s, f)
            F_ref, tau_ref, _ = o.forces_torques(f, Gn @ s_ref)
            assert np.abs(F - F_ref).max() < 1e-9 * np.abs(F_ref).max()
            assert np.abs(tau - tau_ref).max() < 1e-9 * max(np.abs(tau_ref).max(), np.abs(F_ref).max())
    finally:
        ctx.close()


def test_batch_refuses_bad_arguments(yk):
    ctx, ctx2 = yk.Context(0), yk.Context(0)
    try:
        wl = W.small_system(2, 73, n_panels=8)
        g = yk.Geometry(ctx, wl.particles, yk.params_for(wl))
        g2 = yk.Geometry(ctx2, wl.particles, yk.params_for(wl))
        f = g.yk_label(yk.YK_LABEL_TANH, 10.0)
        for geoms in ([g, g], [g, g2]):
            with pytest.raises(yk.YKError) as e:
                yk.yk_solve_batch(geoms, [f, f])
            assert e.value.code == yk.YK_ERR_ARG
    finally:
        ctx.close()
        ctx2.close()
