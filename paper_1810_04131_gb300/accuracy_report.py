"""Accuracy and speed of the mixed-precision solver against the FP64 path on
the 512-ellipse system (semi-axes 1.0 x 0.5, 200 x 200 box, gap >= 0.2,
16 panels x 16 nodes, QBX order 10), for screening lengths rho in
{0.25, 1, 4}.

For each rho: one FP64 solve to a 1e-12 residual (the reference), one mixed
solve to --mixed-tol (default 1e-11: forces and torques carry about 60 times
the density error at rho = 4, so this keeps them a factor of ten inside the
1e-9 bar), and the relative errors of the mixed density, off-surface
potential (200 targets at least 0.25 from every boundary), forces and
torques against it. The FP64 oracle recomputes the residual of both
densities at sampled rows, an independent check at full size.

    python -m paper_1810_04131_gb300.accuracy_report [--rhos 0.25 1 4] [--mixed-tol 1e-11] [--json out.json]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rhos", type=float, nargs="+", default=[0.25, 1.0, 4.0])
    ap.add_argument("--oracle-rows", type=int, default=24)
    ap.add_argument("--mixed-tol", type=float, default=1e-11)
    ap.add_argument("--json", default=None)
    a = ap.parse_args()
    import torch
    from paper_1810_04131_gb300 import workloads as W
    from paper_1810_04131_gb300 import yk
    torch.cuda.set_device(0)
    ctx = yk.Context(0)
    base = W.ellipses512()
    targets = W.off_surface_targets(base.particles, 200, base.box, 0.25, seed=8)
    rows = []
    for rho in a.rhos:
        wl = W.ellipses512(rho)
        res = {"rho": rho}
        out = {}
        for name, prec, tol in (("fp64", yk.YK_FP64, 1e-12), ("mixed", yk.YK_MIXED, a.mixed_tol)):
            g = yk.Geometry(ctx, wl.particles, yk.params_for(wl, precision=prec, gmres_tol=tol,
                                                             max_iter=400))
            f = g.yk_label(yk.YK_LABEL_TANH, 10.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sig, F, tau, info = g.yk_solve_forces(f)
            t = time.perf_counter() - t0
            u = g.yk_eval_potential(sig, targets)
            out[name] = dict(sigma=sig, F=F.reshape(-1, 2), tau=tau, u=u, f=f, info=info, t=t)
            g.close()
        ref, mix = out["fp64"], out["mixed"]
        rel = lambda x, y: float(np.linalg.norm(x - y) / np.linalg.norm(y))
        res.update(
            fp64_s=ref["t"], mixed_s=mix["t"], speedup=ref["t"] / mix["t"],
            fp64_iters=ref["info"]["iterations"], mixed_iters=mix["info"]["iterations"],
            mixed_refinements=mix["info"]["refinements"],
            mixed_residual=mix["info"]["rel_residual"],
            err_sigma=rel(mix["sigma"], ref["sigma"]), err_u=rel(mix["u"], ref["u"]),
            err_F=float(np.abs(mix["F"] - ref["F"]).max() / np.abs(ref["F"]).max()),
            err_tau=float(np.abs(mix["tau"] - ref["tau"]).max() / np.abs(ref["tau"]).max()),
            max_F=float(np.abs(ref["F"]).max()))
        if a.oracle_rows > 0:
            from oracle import yk_oracle as yo
            o = yo.Oracle(wl.particles, wl.n_panels, wl.n_gl, wl.rho,
                          yo.QBXParams(order=wl.qbx_order))
            rng = np.random.default_rng(1)
            idx = np.sort(rng.choice(len(ref["f"]), a.oracle_rows, replace=False))
            fmax = np.abs(ref["f"]).max()
            for name in ("fp64", "mixed"):
                r = ref["f"][idx] - o.apply_rows(out[name]["sigma"], idx)
                res["oracle_residual_%s" % name] = float(np.abs(r).max() / fmax)
        rows.append(res)
        print(json.dumps(res), flush=True)
    ctx.close()
    if a.json:
        json.dump(rows, open(a.json, "w"), indent=1)


if __name__ == "__main__":
    main()
