"""The stored oracle reference solutions (tests/golden/ref_<workload>.npz),
checked on the CPU against the oracle and the seeded inputs they claim.

Each file holds the oracle's solution of one seeded system (Eq. bie), its
normal derivative and its forces and torques (Eqs. stress, force_torque,
scalar-torque), written by tests/golden/make_reference_solution.py. Here:
  * the metadata: GMRES run to 1e-13, true residual below 1e-12;
  * the particles equal the seeded placement of the named workload (and
    the hash recorded when the file was written);
  * the data f equals the oracle's tanh label on those particles;
  * the stored density solves the oracle's operator at sampled rows
    (f_i - (A sigma)_i, with A the oracle's own rows), so the file belongs
    to this oracle and this system;
  * forces and torques sum to nearly zero (Eq. net), relative to the sum
    of the absolute stress contributions (the residue is the
    discretisation error of the steep tanh label on 16 x 16 nodes).
"""
import glob
import hashlib
import os
import sys

import numpy as np
import pytest

from oracle import yk_oracle as yo
from paper_1810_04131_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
sys.path.insert(0, GOLDEN)
from make_reference_solution import read_meta  # noqa: E402

REFS = sorted(os.path.basename(p)[4:-4] for p in glob.glob(os.path.join(GOLDEN, "ref_*.npz")))


def workload(name):
    if name.startswith("ellipses512_rho"):
        return W.ellipses512(float(name[len("ellipses512_rho"):]))
    if name.startswith("ellipses128_rho"):
        return W.ellipses128(float(name[len("ellipses128_rho"):]))
    return W.WORKLOADS[name]()


@pytest.mark.parametrize("name", REFS)
def test_reference_solution(name):
    z = np.load(os.path.join(GOLDEN, "ref_%s.npz" % name))
    meta = read_meta(z)
    wl = workload(name)
    assert meta["workload"] == wl.name == name
    assert meta["tol"] <= 1e-13 and meta["rel_residual_true"] <= 1e-12
    assert np.array_equal(z["particles"], wl.particles)
    assert hashlib.sha256(np.ascontiguousarray(wl.particles).tobytes()).hexdigest() == \
        meta["particles_sha256"]
    o = yo.Oracle(wl.particles, wl.n_panels, wl.n_gl, wl.rho, yo.QBXParams(order=wl.qbx_order))
    n = o.geom.n
    assert z["sigma"].shape == (n,) and z["F"].shape == (wl.n_particles, 2)
    assert z["tau"].shape == (wl.n_particles,)
    f = yo.label(o.geom, wl.label_kind, wl.label_param)
    assert np.array_equal(f, z["f"])
    rows = np.sort(np.random.default_rng(5).choice(n, 6, replace=False))
    r = f[rows] - o.apply_rows(z["sigma"], rows)
    assert np.abs(r).max() <= 1e-11 * np.abs(f).max(), np.abs(r).max()
    # Eq. net against the size of the stress integrand (Eq. stress from the
    # stored f and u_nu): the net force and torque are 1e-7 to 1e-6 of it,
    # the discretisation error of the steep label on 16 x 16 nodes
    g = o.geom
    ut = o.tangential_derivative(f)
    un = z["u_nu"]
    Tn = ((f * f / wl.rho + wl.rho * (ut * ut - un * un))[:, None] * g.nu
          - (2.0 * wl.rho * un * ut)[:, None] * g.tau)
    F, tau0 = z["F"], z["tau0"]
    assert np.abs(F.sum(0)).max() <= 2e-6 * (g.w[:, None] * np.abs(Tn)).sum()
    lever = np.abs(g.x[:, 0] * Tn[:, 1] - g.x[:, 1] * Tn[:, 0])
    assert abs(tau0.sum()) <= 2e-6 * (g.w * lever).sum()
    # the torque about the centres from the torque about the origin
    a = wl.particles[:, 1:3]
    assert np.allclose(z["tau"], tau0 - (a[:, 0] * F[:, 1] - a[:, 1] * F[:, 0]), rtol=0, atol=1e-12)
