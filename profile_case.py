"""Run one kernel case of the yk library on a named workload, for profilers.

    python profile_case.py --case p2p_f32 --workload disks512 --reps 2
        [--farfield dense|cutoff|fmm] [--particles K]

Cases: p2p_f32 (mixed matvec: FP32 far field + near rows), p2p_f64 (FP64
matvec), grad (precision-split normal derivative), qbx (geometry + QBX rows), solve (one mixed solve +
forces), stokes_f64 / stokes_f32 (the Stokes mobility operator, FP64 with
particle expansions / FP32), mobility (one mixed Stokes mobility solve under
unit loads). Workloads: the named ones and table2_<n> (n = 250, 500, 1000,
2000). The geometry is built first; then the case runs --reps times. The case
requests instead solves single requests of the seeded serving stream alone (one
of about 4, 6, 13, 34, 68 and 156 particles), twice each, and prints the wall
time of geometry creation and of the second solve.
--particles K keeps the first K particles of the workload (a smaller case of
the same kernels, for captures that replay each launch many times).
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="p2p_f32",
                    choices=["p2p_f32", "p2p_f64", "grad", "qbx", "solve", "requests",
                             "stokes_f64", "stokes_f32", "mobility"])
    ap.add_argument("--workload", default="disks512")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--farfield", default="dense", choices=["dense", "cutoff", "fmm"])
    ap.add_argument("--particles", type=int, default=0)
    a = ap.parse_args()
    import torch
    from paper_1810_04131_gb300 import workloads as W
    from paper_1810_04131_gb300 import yk
    if a.case == "requests":
        return requests(torch, W, yk)
    if a.workload.startswith("table2_"):
        wl = W.table2(int(a.workload[len("table2_"):]))
    else:
        wl = W.WORKLOADS[a.workload]()
    if a.particles > 0:
        wl.particles = wl.particles[:a.particles]
    ctx = yk.Context(0, torch.cuda.current_stream().cuda_stream)
    prm = yk.params_for(wl, farfield={"dense": yk.YK_FARFIELD_DENSE,
                                      "cutoff": yk.YK_FARFIELD_CUTOFF,
                                      "fmm": yk.YK_FARFIELD_FMM}[a.farfield])
    g = yk.Geometry(ctx, wl.particles, prm)
    dev = torch.device("cuda", 0)
    f = torch.zeros(g.n, dtype=torch.float64, device=dev)
    g.yk_label(yk.YK_LABEL_TANH, 10.0, out=f)
    y = torch.zeros_like(f)
    for _ in range(a.reps):
        if a.case == "p2p_f32":
            g.yk_matvec(f, yk.YK_MIXED, out=y)
        elif a.case == "p2p_f64":
            g.yk_matvec(f, yk.YK_FP64, out=y)
        elif a.case == "grad":
            g.yk_normal_derivative(f, yk.YK_MIXED, out=y)
        elif a.case == "qbx":
            g2 = yk.Geometry(ctx, wl.particles, prm)
            g2.close()
        elif a.case in ("stokes_f64", "stokes_f32"):
            s2 = torch.ones(2 * g.n, dtype=torch.float64, device=dev)
            o2 = torch.zeros_like(s2)
            g.yk_stokes_apply(s2, yk.YK_STOKES_COMPLETED,
                              yk.YK_FP64 if a.case == "stokes_f64" else yk.YK_MIXED, out=o2)
        elif a.case == "mobility":
            n = g.n_particles
            g.yk_mobility([[1.0, 0.0]] * n, [0.5] * n)
        elif a.case == "solve":
            s, info = g.yk_solve(f, out=y)
            g.yk_forces_torques(y, f, want_net=False)
    torch.cuda.synchronize()
    print("ok", a.case, a.workload, g.n)
    g.close()
    ctx.close()


def requests(torch, W, yk):
    """Single requests of the seeded stream, each solved alone."""
    import time
    ctx = yk.Context(0)
    stream = W.request_stream(200, seed=6, rate=1.0)
    for target in (4, 6, 13, 34, 68, 156):
        r = min(stream, key=lambda q: abs(q["n_particles"] - target))
        wl = W.materialise_request(r)
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = yk.Geometry(ctx, wl.particles, yk.params_for(wl, precision=yk.YK_MIXED))
            torch.cuda.synchronize()
            t_create = time.perf_counter() - t0
            f = g.yk_label(yk.YK_LABEL_TANH, 10.0)
            g.yk_solve_forces(f)
            t0 = time.perf_counter()
            s, F, tau, info = g.yk_solve_forces(f)
            t_solve = time.perf_counter() - t0
            g.close()
        print("particles %d panels %d nodes %d: create %.2f ms, solve %.2f ms (%d iterations, "
              "%d refinements)" % (wl.n_particles, wl.n_panels, wl.n_nodes, t_create * 1e3,
                                   t_solve * 1e3, info["iterations"], info["refinements"]))
    ctx.close()


if __name__ == "__main__":
    main()
