"""Seeded synthetic particle configurations (inputs only).

This module draws particle systems: centres, orientations and semi-axes,
with a minimum surface gap between particles. It holds none of the method's
arithmetic (no discretisation, no kernel, no solve), so both the CUDA path
and the FP64 oracle read their inputs from here.

The paper measures on randomly generated, non-overlapping unit disks in a
square box (Section 6.3, Table 2) and on Janus ellipses (Section 2.1). The
named workloads below follow that recipe with the sizes of the benchmark
configurations:

  * ``disks8``    8 unit disks in a 20x20 box, gap >= 0.5, 16x16 nodes, rho=1, QBX order 8.
  * ``disks512``  512 unit disks in a 200x200 box, gap >= 0.3, 16x16 nodes, rho=1, QBX order 10.
  * ``ellipses512`` 512 ellipses 1.0x0.5 in a 200x200 box, gap >= 0.2, 16x16 nodes, QBX order 10.
  * ``ellipses128`` 128 such ellipses in a 100x100 box (same area fraction), N = 32768.
  * ``disks8192`` 8192 unit disks in an 800x800 box, gap >= 0.3, 16x16 nodes.
  * ``stream``    seeded request stream (Poisson arrivals, log-uniform sizes).

A particle row is ``(shape, cx, cy, phi, A, B)`` with shape 0 = disk and
1 = ellipse; A is the semi-axis along the director d = (cos phi, sin phi)
and B the one across it (A = B = radius for a disk).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SHAPE_DISK = 0
SHAPE_ELLIPSE = 1

# label kinds (Dirichlet data generators); values match the C header
LABEL_TANH = 0     # f = (1 + tanh(param * cos(theta - phi))) / 2
LABEL_SINP = 1     # f = 1 - sin^param(theta - phi)          (Eq. JanusBC)
LABEL_COS = 2      # f = (1 + cos(theta - phi)) / 2          (the analytic test of Eq. true_soln)
LABEL_CUSTOM = 3


def _boundary_samples(p, m=4096):
    """Dense boundary points of one particle row (for gap checks only)."""
    t = np.linspace(0.0, 2.0 * np.pi, m, endpoint=False)
    c, s = math.cos(p[3]), math.sin(p[3])
    u = p[4] * np.cos(t)
    v = p[5] * np.sin(t)
    return np.stack([p[1] + c * u - s * v, p[2] + s * u + c * v], axis=1)


def _gap_at_least(p, q, gap):
    """Whether the surface gap of two particles (disks exact; ellipses as the
    smallest distance between 4096 samples of p's boundary and every fourth of
    4096 samples of q's) is at least ``gap``.

    Bounding circles at least gap apart accept at once (every sampled
    distance is at least theirs). Otherwise the samples are grouped around
    every 16th one: a sample lies within 8 sample steps, so within
    8 (2 pi max(A, B) / 4096) of its group's centre, and a pair of groups
    whose centres are d apart holds no sampled pair closer than d minus both
    bounds. Only the groups that could hold a pair closer than gap are
    compared sample by sample, which gives exactly the answer of comparing
    all of them."""
    d = math.hypot(p[1] - q[1], p[2] - q[2])
    if p[0] == SHAPE_DISK and q[0] == SHAPE_DISK:
        return d - p[4] - q[4] >= gap
    ra, rb = max(p[4], p[5]), max(q[4], q[5])
    if d - ra - rb >= gap:   # bounding circles: every boundary distance is at least this
        return True
    a, b = _boundary_samples(p), _boundary_samples(q)
    m = a.shape[0]
    dc = np.sqrt(((a[::16, None, :] - b[None, ::16, :]) ** 2).sum(-1))
    if dc.min() < gap:       # group centres are samples themselves
        return False
    slack = 8.0 * 2.0 * math.pi * (ra + rb) / m
    gi, gj = np.nonzero(dc - slack < gap)
    if gi.size == 0:
        return True
    ia = (16 * gi[:, None] + np.arange(-8, 9)[None, :]) % m          # p's samples
    jb = (16 * gj[:, None] + np.arange(-8, 9, 4)[None, :]) % m       # q's, every fourth
    diff = a[ia][:, :, None, :] - b[jb][:, None, :, :]
    return bool(np.sqrt((diff ** 2).sum(-1)).min() >= gap)


_PLACED = {}


def make_particles(n, box, gap, seed, shape=SHAPE_DISK, A=1.0, B=1.0,
                   shapes=None, max_tries=2_000_000):
    """Rejection-sample ``n`` non-overlapping particles in ``[0, box]^2``
    (memoised per process: the same arguments return a copy of the same
    array)."""
    key = (n, box, gap, seed, shape, A, B, None if shapes is None else tuple(shapes), max_tries)
    if key not in _PLACED:
        _PLACED[key] = _place(n, box, gap, seed, shape, A, B, shapes, max_tries)
    return _PLACED[key].copy()


def _place(n, box, gap, seed, shape, A, B, shapes, max_tries):
    """Rejection-sample ``n`` non-overlapping particles in ``[0, box]^2``.

    Centres are uniform in ``[R, box - R]^2`` (R = max semi-axis) and a
    candidate is accepted when its surface gap to every accepted particle is
    at least ``gap``; orientations are uniform in ``[0, 2 pi)``. ``shapes``
    optionally gives a per-particle shape list (0 disk / 1 ellipse).
    Returns a float64 array of shape (n, 6).
    """
    rng = np.random.default_rng(seed)
    out = np.zeros((n, 6))
    R = max(A, B)
    cell = 2.0 * R + gap
    grid = {}
    k = 0
    tries = 0
    while k < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place %d particles (placed %d)" % (n, k))
        cx, cy = rng.uniform(R, box - R, size=2)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        sh = shape if shapes is None else shapes[k]
        a_, b_ = (A, B) if sh == SHAPE_ELLIPSE else (A, A)
        cand = np.array([sh, cx, cy, phi, a_, b_])
        gx, gy = int(cx // cell), int(cy // cell)
        ok = True
        for ix in range(gx - 1, gx + 2):
            for iy in range(gy - 1, gy + 2):
                for j in grid.get((ix, iy), ()):
                    if not _gap_at_least(cand, out[j], gap):
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            out[k] = cand
            grid.setdefault((gx, gy), []).append(k)
            k += 1
    return out


def off_surface_targets(particles, nt, box, min_dist, seed):
    """``nt`` seeded targets uniform in ``[0, box]^2``, outside every particle
    and at least ``min_dist`` from every boundary."""
    rng = np.random.default_rng(seed)
    pts = []
    samples = [_boundary_samples(p) for p in particles]
    while len(pts) < nt:
        t = rng.uniform(0.0, box, size=2)
        ok = True
        for p, s in zip(particles, samples):
            d = math.hypot(t[0] - p[1], t[1] - p[2])
            if d > max(p[4], p[5]) + min_dist + 0.01:
                continue
            # inside test in the particle frame, then sampled distance
            c, sn = math.cos(p[3]), math.sin(p[3])
            u = c * (t[0] - p[1]) + sn * (t[1] - p[2])
            v = -sn * (t[0] - p[1]) + c * (t[1] - p[2])
            if (u / p[4]) ** 2 + (v / p[5]) ** 2 <= 1.0:
                ok = False
                break
            if np.sqrt(((s - t) ** 2).sum(-1)).min() < min_dist:
                ok = False
                break
        if ok:
            pts.append(t)
    return np.array(pts)


@dataclass
class Workload:
    """A named synthetic system: particles plus the numerical parameters."""
    name: str
    particles: np.ndarray
    rho: float
    n_panels: int = 16
    n_gl: int = 16
    qbx_order: int = 10
    gmres_tol: float = 1e-12
    label_kind: int = LABEL_TANH
    label_param: float = 10.0
    box: float = 0.0
    targets: np.ndarray | None = None
    extra: dict = field(default_factory=dict)

    @property
    def n_particles(self):
        return int(self.particles.shape[0])

    @property
    def n_nodes(self):
        return self.n_particles * self.n_panels * self.n_gl


def disks8():
    """8 unit disks, 20x20 box, gap 0.5, N = 2048, rho = 1, QBX order 8."""
    p = make_particles(8, 20.0, 0.5, seed=1)
    t = off_surface_targets(p, 1000, 20.0, 0.25, seed=2)
    return Workload("disks8", p, rho=1.0, qbx_order=8, box=20.0, targets=t)


def disks512():
    """512 unit disks, 200x200 box, gap 0.3, N = 131072, rho = 1, QBX order 10."""
    p = make_particles(512, 200.0, 0.3, seed=3)
    return Workload("disks512", p, rho=1.0, qbx_order=10, box=200.0)


def ellipses512(rho=1.0):
    """512 ellipses 1.0x0.5, 200x200 box, gap 0.2, N = 131072, QBX order 10."""
    p = make_particles(512, 200.0, 0.2, seed=4, shape=SHAPE_ELLIPSE, A=1.0, B=0.5)
    return Workload("ellipses512_rho%g" % rho, p, rho=rho, qbx_order=10, box=200.0)


def ellipses128(rho=1.0):
    """128 ellipses 1.0x0.5 in a 100x100 box (the area fraction of ``ellipses512``),
    gap 0.2, N = 32768, QBX order 10: the ellipse system at which the FP64 oracle
    finishes a full solve for every screening length in minutes."""
    p = make_particles(128, 100.0, 0.2, seed=7, shape=SHAPE_ELLIPSE, A=1.0, B=0.5)
    return Workload("ellipses128_rho%g" % rho, p, rho=rho, qbx_order=10, box=100.0)


def disks8192():
    """8192 unit disks, 800x800 box, gap 0.3, N = 2,097,152, rho = 1."""
    p = make_particles(8192, 800.0, 0.3, seed=5)
    return Workload("disks8192", p, rho=1.0, qbx_order=10, box=800.0)


TABLE2_BOX = {250: 100.0, 500: 200.0, 1000: 200.0, 2000: 400.0}


def table2(n_particles):
    """The large collections of Table 2: n unit disks in the printed L x L box
    (250: 100, 500 and 1000: 200, 2000: 400), 70 boundary points per particle
    (10 panels x 7 nodes, the N_GL = 7 reading of Table 1), rho = 4, GMRES
    tolerance 1e-5 as printed. Not printed, taken here: QBX order 8 (Table 1's
    highest at 70 points) and a minimum gap of 0.5."""
    box = TABLE2_BOX[n_particles]
    p = make_particles(n_particles, box, 0.5, seed=20 + n_particles)
    return Workload("table2_%d" % n_particles, p, rho=4.0, n_panels=10, n_gl=7, qbx_order=8,
                    gmres_tol=1e-5, box=box)


def small_system(n, seed, shape=SHAPE_DISK, n_panels=8, n_gl=16, rho=1.0,
                 qbx_order=10, gap=0.5, A=1.0, B=1.0):
    """A small seeded system for parity tests (box scaled to ~4% area fraction)."""
    R = max(A, B)
    box = max(4.0 * R + gap, math.sqrt(n * math.pi * R * R / 0.04))
    p = make_particles(n, box, gap, seed=seed, shape=shape, A=A, B=B)
    return Workload("small%d_s%d" % (n, seed), p, rho=rho, n_panels=n_panels,
                    n_gl=n_gl, qbx_order=qbx_order, box=box)


def request_stream(n_requests=2000, seed=6, rate=None, np_min=4, np_max=2048,
                   pan_min=8, pan_max=32, rhos=(0.5, 1.0, 2.0), gap=0.3):
    """Seeded serving stream: Poisson arrivals, log-uniform particle counts,
    panels per particle uniform in [pan_min, pan_max], disk/ellipse 50/50,
    rho from ``rhos``, box side 200*sqrt(Np/512) (about 4% area fraction).

    Returns a list of dicts with the request parameters; the particles are
    drawn lazily by ``materialise_request`` so that a long stream stays cheap.
    """
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for i in range(n_requests):
        if rate:
            t += rng.exponential(1.0 / rate)
        npart = int(round(math.exp(rng.uniform(math.log(np_min), math.log(np_max)))))
        npan = int(rng.integers(pan_min, pan_max + 1))
        shape = int(rng.integers(0, 2))
        rho = float(rhos[int(rng.integers(0, len(rhos)))])
        box = max(8.0, 200.0 * math.sqrt(npart / 512.0))
        reqs.append(dict(id=i, arrival=t, n_particles=npart, n_panels=npan,
                         shape=shape, rho=rho, box=box, gap=gap,
                         seed=int(rng.integers(0, 2 ** 31 - 1))))
    return reqs


def materialise_request(r):
    """Draw the particles of one stream request."""
    A, B = (1.0, 0.5) if r["shape"] == SHAPE_ELLIPSE else (1.0, 1.0)
    p = make_particles(r["n_particles"], r["box"], r["gap"], seed=r["seed"],
                       shape=r["shape"], A=A, B=B)
    return Workload("req%d" % r["id"], p, rho=r["rho"], n_panels=r["n_panels"],
                    qbx_order=10, box=r["box"])


WORKLOADS = {
    "disks8": disks8,
    "disks512": disks512,
    "ellipses512": ellipses512,
    "ellipses128": ellipses128,
    "disks8192": disks8192,
}
