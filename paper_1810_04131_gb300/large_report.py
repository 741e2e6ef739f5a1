"""The large system: 8192 unit disks in an 800 x 800 box (gap >= 0.3,
16 panels x 16 nodes, N = 2,097,152, rho = 1, QBX order 10) with the cut-off
far field (source particles whose contribution is bounded below
cutoff_tol * max|sigma| are left out; default 1e-15) and with the FMM far
field for the inner operator (order 12, leaf size autotuned).

Reports each mixed-precision solve (label, GMRES with FP64 refinement,
forces) and the FP64 solve with the cut-off far field, their agreement, and
an independent check against the FP64 oracle: the dense operator (every
source, no cut-off) at sampled rows, applied to the GPU densities.

    python -m paper_1810_04131_gb300.large_report [--fp64 1] [--oracle-rows 12]
        [--farfields cutoff fmm]
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
    ap.add_argument("--fp64", type=int, default=1)
    ap.add_argument("--oracle-rows", type=int, default=12)
    ap.add_argument("--json", default=None)
    ap.add_argument("--farfields", nargs="+", default=["cutoff", "fmm"])
    a = ap.parse_args()
    import torch
    from paper_1810_04131_gb300 import workloads as W
    from paper_1810_04131_gb300 import yk
    torch.cuda.set_device(0)
    wl = W.disks8192()
    ctx = yk.Context(0, torch.cuda.current_stream().cuda_stream)
    res = {"workload": "disks8192", "n_nodes": wl.n_nodes, "cutoff_tol": 1e-15, "fmm_order": 12}
    out = {}
    ff = {"cutoff": yk.YK_FARFIELD_CUTOFF, "fmm": yk.YK_FARFIELD_FMM}
    modes = [("mixed" if f == "cutoff" else "mixed_" + f, yk.YK_MIXED, ff[f]) for f in a.farfields]
    modes += [("fp64", yk.YK_FP64, yk.YK_FARFIELD_CUTOFF)] if a.fp64 else []
    for name, prec, farfield in modes:
        # the FP64 solve is the reference: run it to a 1e-12 residual
        tol = 1e-12 if prec == yk.YK_FP64 else wl.gmres_tol
        g = yk.Geometry(ctx, wl.particles, yk.params_for(wl, precision=prec, gmres_tol=tol,
                                                         farfield=farfield))
        dev = torch.device("cuda", 0)
        f = torch.zeros(g.n, dtype=torch.float64, device=dev)
        sig = torch.zeros_like(f)
        F = torch.zeros((g.n_particles, 2), dtype=torch.float64, device=dev)
        tau = torch.zeros(g.n_particles, dtype=torch.float64, device=dev)
        reps = 2 if name.startswith("mixed") else 1
        times = []
        for _ in range(reps):   # the first mixed solve also builds lists and tunes the FMM
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.yk_update_geometry(wl.particles)
            g.yk_label(yk.YK_LABEL_TANH, 10.0, out=f)
            _, info = g.yk_solve(f, out=sig)
            g.yk_forces_torques(sig, f, F=F, tau=tau, want_net=False)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        res["%s_solve_s" % name] = times[-1]
        res["%s_first_solve_s" % name] = times[0]
        res["%s_info" % name] = info
        out[name] = dict(sigma=sig.cpu().numpy(), F=F.cpu().numpy(), f=f.cpu().numpy())
        if name.startswith("mixed"):
            y = torch.zeros_like(f)
            g.yk_matvec(sig, yk.YK_MIXED, out=y)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(5):
                g.yk_matvec(sig, yk.YK_MIXED, out=y)
            torch.cuda.synchronize()
            res["%s_matvec_ms" % name] = (time.perf_counter() - t0) / 5 * 1e3
        if name == "mixed":
            y64 = torch.zeros_like(f)
            g.yk_matvec(sig, yk.YK_FP64, out=y64)
            out["y64"] = y64.cpu().numpy()
            out["sig_for_y64"] = sig.cpu().numpy()
        g.close()
        print(json.dumps({k: v for k, v in res.items()}), flush=True)
    for name in [k for k in out if k.startswith("mixed") and "fp64" in out]:
        m, r = out[name], out["fp64"]
        res["sigma_rel_diff_%s_vs_fp64" % name] = float(np.linalg.norm(m["sigma"] - r["sigma"]) /
                                                       np.linalg.norm(r["sigma"]))
        res["F_rel_diff_%s_vs_fp64" % name] = float(np.abs(m["F"] - r["F"]).max() /
                                                    np.abs(r["F"]).max())
        res["speedup_%s_vs_fp64" % name] = res["fp64_solve_s"] / res["%s_solve_s" % name]
    if a.oracle_rows > 0:
        from oracle import yk_oracle as yo
        o = yo.Oracle(wl.particles, wl.n_panels, wl.n_gl, wl.rho, yo.QBXParams(order=wl.qbx_order))
        rng = np.random.default_rng(2)
        rows = np.sort(rng.choice(wl.n_nodes, a.oracle_rows, replace=False))
        if "y64" in out:
            ref = o.apply_rows(out["sig_for_y64"], rows)       # dense, every source
            res["fp64_cutoff_vs_dense_oracle_rows_rel"] = float(
                np.abs(out["y64"][rows] - ref).max() / np.abs(ref).max())
        for name in [k for k in out if k.startswith("mixed")]:
            f = out[name]["f"]
            r = f[rows] - o.apply_rows(out[name]["sigma"], rows)
            res["oracle_residual_%s_rows" % name] = float(np.abs(r).max() / np.abs(f).max())
    ctx.close()
    print(json.dumps(res), flush=True)
    if a.json:
        json.dump(res, open(a.json, "w"), indent=1)


if __name__ == "__main__":
    main()
