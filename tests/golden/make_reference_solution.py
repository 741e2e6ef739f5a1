"""Write the FP64 oracle's reference solution of a full benchmark system.

Test infrastructure: calls only ``oracle/`` (and the seeded placement in
``workloads``, which holds no arithmetic of the method). Nothing here touches
the CUDA library. The output ``ref_<workload>.npz`` is the parity reference
that the GPU tests compare the library's default solves against.

What it computes for one seeded system (Eq. bie and Eqs. stress,
force_torque, scalar-torque):
  * f: the tanh Janus label (Eq. JanusBC family) from ``yk_oracle.label``;
  * sigma: the solution of (1/2 I + D) sigma = f, where every application of
    the operator is ``Oracle.apply_rows`` (plain quadrature far, one-sided QBX
    near) and the Krylov solver is ``Oracle.gmres`` run to a relative
    residual of ``--tol`` (default 1e-13);
  * u_nu from ``Oracle.apply_rows(..., want_grad=True)`` and F, tau from
    ``Oracle.forces_torques``.

Two choices that change the cost, not the result:
  * rows are spread over a process pool (spawn start method, one ``Oracle``
    per worker); each row is still evaluated by the oracle's own row code;
  * GMRES runs on the right-preconditioned operator A M^-1 with M the
    block diagonal of A (every particle's own 256 x 256 interaction block,
    assembled by ``Oracle.dense`` on that particle alone). With right
    preconditioning the residual GMRES drives down is f - A sigma itself,
    so the stopping rule and the solution are those of the unpreconditioned
    system; M only cuts the number of full-size operator applications.
After the solve the true residual ||f - A sigma|| / ||f|| is recomputed with
one more full operator application and stored beside the result.

Usage (hours of CPU at N = 131,072):
    python tests/golden/make_reference_solution.py disks512
    python tests/golden/make_reference_solution.py ellipses512 --rho 4
    python tests/golden/make_reference_solution.py ellipses128 --rho 0.25   (N = 32,768)
"""
from __future__ import annotations

import argparse
import ast
import hashlib
import json
import multiprocessing as mp
import re
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

_ORC = None


def _init(particles, n_panels, n_gl, rho, order):
    global _ORC
    from oracle import yk_oracle as yo
    _ORC = yo.Oracle(particles, n_panels, n_gl, rho, yo.QBXParams(order=order))


def _rows(args):
    sigma, lo, hi, want_grad = args
    out = _ORC.apply_rows(sigma, range(lo, hi), want_grad=want_grad)
    return lo, out


def _self_block(args):
    """Own-particle block of particle i: the oracle's dense operator of the
    particle alone (its near rows by QBX, its own far pairs by quadrature;
    other particles never enter a particle's own block)."""
    from oracle import yk_oracle as yo
    row, n_panels, n_gl, rho, order = args
    o = yo.Oracle(row[None, :], n_panels, n_gl, rho, yo.QBXParams(order=order))
    return np.linalg.inv(o.dense())


def read_meta(z):
    """The metadata dictionary of a stored reference (JSON; files written
    before the switch to JSON hold a Python repr with numpy scalars)."""
    text = str(z["meta"])
    try:
        return json.loads(text)
    except ValueError:
        return ast.literal_eval(re.sub(r"np\.float64\(([^)]*)\)", r"\1", text))


class PooledOperator:
    def __init__(self, pool, n, chunks):
        self.pool = pool
        self.n = n
        edges = np.linspace(0, n, chunks + 1).astype(int)
        self.ranges = [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]
        self.applications = 0
        self.seconds = 0.0

    def apply(self, sigma, want_grad=False):
        t0 = time.time()
        y = np.zeros(self.n)
        yn = np.zeros(self.n) if want_grad else None
        tasks = [(sigma, a, b, want_grad) for a, b in self.ranges]
        for lo, out in self.pool.imap_unordered(_rows, tasks):
            if want_grad:
                y[lo:lo + len(out[0])] = out[0]
                yn[lo:lo + len(out[1])] = out[1]
            else:
                y[lo:lo + len(out)] = out
        self.applications += 1
        self.seconds += time.time() - t0
        return (y, yn) if want_grad else y


def workload(name, rho):
    from paper_1810_04131_gb300 import workloads as W
    if name in ("ellipses512", "ellipses128"):
        return W.WORKLOADS[name](rho)
    wl = W.WORKLOADS[name]()
    if rho is not None and rho != wl.rho:
        raise SystemExit("%s has rho = %g" % (name, wl.rho))
    return wl


def main():
    from oracle import yk_oracle as yo
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--rho", type=float, default=None)
    ap.add_argument("--tol", type=float, default=1e-13)
    ap.add_argument("--workers", type=int, default=os.cpu_count())
    ap.add_argument("--chunks", type=int, default=0)
    ap.add_argument("--max-iter", type=int, default=200)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    wl = workload(a.workload, a.rho if a.rho is not None else None)
    out = a.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), "ref_%s.npz" % wl.name)
    t_start = time.time()
    orc = yo.Oracle(wl.particles, wl.n_panels, wl.n_gl, wl.rho, yo.QBXParams(order=wl.qbx_order))
    g = orc.geom
    n, npp = g.n, wl.n_panels * wl.n_gl
    f = yo.label(g, wl.label_kind, wl.label_param)
    ctx = mp.get_context("spawn")
    init = (wl.particles, wl.n_panels, wl.n_gl, wl.rho, wl.qbx_order)
    with ctx.Pool(a.workers, initializer=_init, initargs=init) as pool:
        op = PooledOperator(pool, n, a.chunks or 16 * a.workers)
        t0 = time.time()
        blocks = pool.map(_self_block, [(row, wl.n_panels, wl.n_gl, wl.rho, wl.qbx_order)
                                        for row in wl.particles], chunksize=4)
        Minv = np.stack(blocks)
        t_blocks = time.time() - t0
        print("%s: N=%d, %d self blocks in %.0f s" % (wl.name, n, len(blocks), t_blocks), flush=True)

        def precond(v):
            return np.einsum("pij,pj->pi", Minv, v.reshape(-1, npp)).ravel()

        def matvec(v):
            y = op.apply(precond(v))
            print("  application %d: %.0f s" % (op.applications, op.seconds / op.applications),
                  flush=True)
            return y

        yv, iters, rel_gmres = yo.Oracle.gmres(matvec, f, tol=a.tol, max_iter=a.max_iter)
        sigma = precond(yv)
        print("GMRES: %d iterations, estimated residual %.3e" % (iters, rel_gmres), flush=True)
        r = f - op.apply(sigma)
        rel_true = float(np.linalg.norm(r) / np.linalg.norm(f))
        print("true residual %.3e" % rel_true, flush=True)
        _, un = op.apply(sigma, want_grad=True)
    F, tau, tau0 = orc.forces_torques(f, un)
    meta = dict(workload=wl.name, n_particles=wl.n_particles, n_panels=wl.n_panels, n_gl=wl.n_gl,
                rho=wl.rho, qbx_order=wl.qbx_order, label_kind=wl.label_kind,
                label_param=wl.label_param, tol=a.tol, iterations=iters,
                rel_residual_gmres=rel_gmres, rel_residual_true=rel_true,
                operator_applications=op.applications, workers=a.workers,
                host=platform.processor() or platform.machine(),
                wall_s=round(time.time() - t_start, 1),
                particles_sha256=hashlib.sha256(np.ascontiguousarray(wl.particles).tobytes()).hexdigest(),
                script="tests/golden/make_reference_solution.py")
    np.savez_compressed(out, particles=wl.particles, f=f, sigma=sigma, u_nu=un, F=F, tau=tau,
                        tau0=tau0, meta=np.array(json.dumps(meta)))
    print("wrote %s (%s)" % (out, meta), flush=True)


if __name__ == "__main__":
    main()
