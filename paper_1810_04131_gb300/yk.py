"""Python binding of the yk C ABI (include/yk.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does
nothing but convert arguments (numpy arrays, torch tensors, plain numbers)
to pointers and sizes and turn error codes into exceptions. All arithmetic
runs in the CUDA library ``lib/libyk.so``; importing this module on a
machine without the built library raises, so nothing can fall back to a
CPU path.

Arrays may be numpy arrays (host) or CUDA torch tensors (device); the
library detects which per pointer.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libyk.so")

YK_OK = 0
YK_ERR_ARG = -1
YK_ERR_BAD_GEOMETRY = -2
YK_ERR_NO_MEMORY = -3
YK_ERR_NOT_CONVERGED = -4
YK_ERR_TIMEOUT = -5
YK_ERR_CUDA = -6
YK_ERR_NOT_FOUND = -7
YK_ERR_BUSY = -8
YK_ERR_TOO_LARGE = -9

YK_SHAPE_DISK = 0
YK_SHAPE_ELLIPSE = 1
YK_FP64 = 0
YK_MIXED = 1
YK_REP_DOUBLE_LAYER = 0
YK_REP_COMBINED = 1
YK_PRECOND_NONE = 0
YK_PRECOND_BLOCK = 1
YK_COARSE_NONE = 0
YK_COARSE_MODES = 1
YK_FARFIELD_DENSE = 0
YK_FARFIELD_CUTOFF = 1
YK_FARFIELD_FMM = 2
YK_LABEL_TANH = 0
YK_LABEL_SINP = 1
YK_LABEL_COS = 2
YK_LABEL_CUSTOM = 3
YK_STOKES_TRACTION = 0
YK_STOKES_COMPLETED = 1
YK_STOKES_VELOCITY = 2
YK_REQ_QUEUED, YK_REQ_RUNNING, YK_REQ_DONE, YK_REQ_FAILED = 0, 1, 2, 3

# every entry point declared in include/yk.h
EXPORTS = [
    "yk_default_params", "yk_create", "yk_destroy", "yk_create_geometry",
    "yk_destroy_geometry", "yk_update_geometry", "yk_kernel_launches", "yk_num_nodes", "yk_nodes", "yk_label", "yk_matvec",
    "yk_normal_derivative", "yk_solve", "yk_forces_torques", "yk_energy", "yk_eval_potential",
    "yk_eval_potential_noalloc", "yk_eval_potential_near", "yk_repulsion", "yk_default_dynamics", "yk_step",
    "yk_solve_forces", "yk_solve_batch", "yk_submit", "yk_poll", "yk_drain", "yk_fp32_fma_peak",
    "yk_stokes_apply", "yk_mobility", "yk_strerror",
]


class yk_particle(C.Structure):
    _fields_ = [("shape", C.c_int32), ("pad_", C.c_int32), ("cx", C.c_double),
                ("cy", C.c_double), ("phi", C.c_double), ("A", C.c_double), ("B", C.c_double)]


class yk_params(C.Structure):
    _fields_ = [("rho", C.c_double), ("gamma", C.c_double), ("n_panels", C.c_int32),
                ("n_gl", C.c_int32), ("qbx_order", C.c_int32), ("oversample", C.c_int32),
                ("qbx_r_factor", C.c_double), ("near_width", C.c_int32),
                ("gmres_restart", C.c_int32), ("max_iter", C.c_int32),
                ("precision", C.c_int32), ("gmres_tol", C.c_double), ("inner_tol", C.c_double),
                ("max_refine", C.c_int32), ("farfield", C.c_int32), ("split_tol", C.c_double),
                ("grad_split_tol", C.c_double), ("precond", C.c_int32), ("pad_", C.c_int32),
                ("cutoff_tol", C.c_double), ("fmm_order", C.c_int32), ("pad2_", C.c_int32),
                ("fmm_leaf", C.c_double), ("representation", C.c_int32), ("pad3_", C.c_int32),
                ("bw_eta", C.c_double), ("viscosity", C.c_double),
                ("coarse", C.c_int32), ("pad4_", C.c_int32)]


class yk_dynamics(C.Structure):
    _fields_ = [("dt", C.c_double), ("xi_x", C.c_double), ("xi_theta", C.c_double),
                ("c0", C.c_double), ("q", C.c_int32), ("label_kind", C.c_int32),
                ("label_param", C.c_double), ("warm_start", C.c_int32), ("mobility", C.c_int32)]


class yk_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("refinements", C.c_int32),
                ("rel_residual", C.c_double), ("matvecs_fp64", C.c_int32),
                ("matvecs_fp32", C.c_int32), ("coarse_dim", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class YKError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.yk_strerror(code).decode() if _lib is not None else str(code)
        super().__init__("%s failed: %s (%d)" % (where, msg, code))


_lib = None
_exiting = False


@atexit.register
def _stop_calls_at_exit():
    """From interpreter exit on, handles dropped during teardown make no
    library call: the CUDA runtime may already be shut down by then (atexit
    handlers run before the objects still alive are finalised). The driver
    releases what such handles held when the process ends."""
    global _exiting
    _exiting = True


def load(path=LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("yk CUDA library not built: %s (run paper_1810_04131_gb300.build)" % path)
    lib = C.CDLL(path)
    P, I, D, I64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
    sig = {
        "yk_default_params": [C.POINTER(yk_params)],
        "yk_create": [C.POINTER(P), I, P],
        "yk_destroy": [P],
        "yk_create_geometry": [P, C.POINTER(yk_particle), I, C.POINTER(yk_params), C.POINTER(P)],
        "yk_destroy_geometry": [P],
        "yk_update_geometry": [P, C.POINTER(yk_particle), I],
        "yk_kernel_launches": [C.POINTER(C.c_uint64)],
        "yk_num_nodes": [P, C.POINTER(I64)],
        "yk_nodes": [P, P, P, P],
        "yk_label": [P, I, D, P, P],
        "yk_matvec": [P, P, P, I],
        "yk_normal_derivative": [P, P, P, I],
        "yk_solve": [P, P, P, P, C.POINTER(yk_solve_info)],
        "yk_forces_torques": [P, P, P, P, P, P],
        "yk_energy": [P, P, P, P, P],
        "yk_repulsion": [P, D, I, P, P, P],
        "yk_default_dynamics": [C.POINTER(yk_dynamics)],
        "yk_step": [P, C.POINTER(yk_dynamics), I, P, P, P],
        "yk_eval_potential": [P, P, P, I64, P],
        "yk_eval_potential_near": [P, P, P, I64, P],
        "yk_eval_potential_noalloc": [P, P, P, I64, P],
        "yk_solve_forces": [P, P, P, P, P, C.POINTER(yk_solve_info)],
        "yk_submit": [P, C.POINTER(yk_particle), I, C.POINTER(yk_params), I, D,
                      C.POINTER(C.c_uint64)],
        "yk_poll": [P, C.c_uint64, C.POINTER(I), P, P, P, C.POINTER(yk_solve_info),
                    C.POINTER(D)],
        "yk_drain": [P],
        "yk_fp32_fma_peak": [I, C.POINTER(D)],
        "yk_solve_batch": [C.POINTER(P), I, C.POINTER(P), C.POINTER(P), P],
        "yk_stokes_apply": [P, I, P, P, I],
        "yk_mobility": [P, P, P, P, P, P, C.POINTER(yk_solve_info)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = I
    lib.yk_strerror.argtypes = [I]
    lib.yk_strerror.restype = C.c_char_p
    _lib = lib
    return lib


def _check(rc, where, ok=(YK_OK,)):
    if rc not in ok:
        raise YKError(rc, where)
    return rc


def _ptr(a):
    """Pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError("expected numpy array or torch tensor, got %r" % type(a))


def _f64(a, n, name):
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or a.size != n:
            raise ValueError("%s: need float64 array of %d elements" % (name, n))
    elif hasattr(a, "dtype"):
        import torch
        if a.dtype != torch.float64 or a.numel() != n:
            raise ValueError("%s: need float64 tensor of %d elements" % (name, n))
    return a


def default_params(**kw):
    p = yk_params()
    load().yk_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def particles_array(rows):
    """(n, 6) array of (shape, cx, cy, phi, A, B) -> ctypes yk_particle array."""
    rows = np.asarray(rows, dtype=np.float64)
    arr = (yk_particle * len(rows))()
    for i, r in enumerate(rows):
        arr[i].shape = int(r[0])
        arr[i].cx, arr[i].cy, arr[i].phi, arr[i].A, arr[i].B = map(float, r[1:6])
    return arr


class Context:
    """yk_create / yk_destroy."""

    def __init__(self, device=0, stream=None):
        lib = load()
        h = C.c_void_p()
        _check(lib.yk_create(C.byref(h), int(device), stream), "yk_create")
        self.h = h
        self.geoms = weakref.WeakSet()

    def close(self):
        if self.h:
            for g in list(self.geoms):   # the C call releases them; drop the handles first
                g.h = None
            load().yk_destroy(self.h)
            self.h = None

    def __del__(self):
        if _exiting:
            return
        try:
            self.close()
        except Exception:
            pass

    # serving
    def yk_submit(self, particles, params, label_kind=YK_LABEL_TANH, label_param=10.0):
        arr = particles_array(particles)
        rid = C.c_uint64()
        _check(load().yk_submit(self.h, arr, len(arr), C.byref(params), int(label_kind),
                                float(label_param), C.byref(rid)), "yk_submit")
        return rid.value

    def yk_poll(self, rid, n_nodes=None, n_particles=None):
        st = C.c_int()
        info = yk_solve_info()
        lat = C.c_double()
        sig = np.zeros(n_nodes) if n_nodes else None
        F = np.zeros(2 * n_particles) if n_particles else None
        tau = np.zeros(n_particles) if n_particles else None
        _check(load().yk_poll(self.h, C.c_uint64(rid), C.byref(st), _ptr(sig), _ptr(F), _ptr(tau),
                              C.byref(info), C.byref(lat)), "yk_poll")
        return dict(status=st.value, sigma=sig, F=F, tau=tau, info=info.as_dict(),
                    latency_ms=lat.value)

    def yk_drain(self):
        _check(load().yk_drain(self.h), "yk_drain")


class Geometry:
    """A discretised configuration (yk_create_geometry / yk_destroy_geometry)."""

    def __init__(self, ctx, particles, params):
        lib = load()
        self.ctx = ctx
        self.params = params
        arr = particles_array(particles)
        self.n_particles = len(arr)
        h = C.c_void_p()
        _check(lib.yk_create_geometry(ctx.h, arr, len(arr), C.byref(params), C.byref(h)),
               "yk_create_geometry")
        self.h = h
        ctx.geoms.add(self)
        n = C.c_int64()
        _check(lib.yk_num_nodes(h, C.byref(n)), "yk_num_nodes")
        self.n = n.value

    def close(self):
        if getattr(self, "h", None):
            load().yk_destroy_geometry(self.h)
            self.h = None

    def __del__(self):
        if _exiting:
            return
        try:
            self.close()
        except Exception:
            pass

    def yk_update_geometry(self, particles):
        arr = particles_array(particles)
        _check(load().yk_update_geometry(self.h, arr, len(arr)), "yk_update_geometry")

    def yk_nodes(self):
        xy = np.zeros((self.n, 2))
        nrm = np.zeros((self.n, 2))
        w = np.zeros(self.n)
        _check(load().yk_nodes(self.h, _ptr(xy), _ptr(nrm), _ptr(w)), "yk_nodes")
        return xy, nrm, w

    def yk_label(self, kind=YK_LABEL_TANH, param=10.0, f_custom=None, out=None):
        out = np.zeros(self.n) if out is None else _f64(out, self.n, "out")
        _check(load().yk_label(self.h, int(kind), float(param), _ptr(f_custom), _ptr(out)),
               "yk_label")
        return out

    def yk_matvec(self, sigma, precision=YK_FP64, out=None):
        _f64(sigma, self.n, "sigma")
        out = np.zeros(self.n) if out is None else _f64(out, self.n, "out")
        _check(load().yk_matvec(self.h, _ptr(sigma), _ptr(out), int(precision)), "yk_matvec")
        return out

    def yk_normal_derivative(self, sigma, precision=YK_FP64, out=None):
        _f64(sigma, self.n, "sigma")
        out = np.zeros(self.n) if out is None else _f64(out, self.n, "out")
        _check(load().yk_normal_derivative(self.h, _ptr(sigma), _ptr(out), int(precision)),
               "yk_normal_derivative")
        return out

    def yk_solve(self, f, sigma0=None, out=None, allow_not_converged=False):
        _f64(f, self.n, "f")
        out = np.zeros(self.n) if out is None else _f64(out, self.n, "out")
        info = yk_solve_info()
        ok = (YK_OK, YK_ERR_NOT_CONVERGED) if allow_not_converged else (YK_OK,)
        rc = _check(load().yk_solve(self.h, _ptr(f), _ptr(out), _ptr(sigma0), C.byref(info)),
                    "yk_solve", ok)
        d = info.as_dict()
        d["converged"] = rc == YK_OK
        return out, d

    def yk_forces_torques(self, sigma, f, F=None, tau=None, want_net=True):
        F = np.zeros((self.n_particles, 2)) if F is None else F
        tau = np.zeros(self.n_particles) if tau is None else tau
        net = np.zeros(3) if want_net else None
        _check(load().yk_forces_torques(self.h, _ptr(sigma), _ptr(f), _ptr(F), _ptr(tau),
                                        _ptr(net)), "yk_forces_torques")
        return F, tau, net

    def yk_energy(self, sigma, f, phi=None):
        """Energy of Eq. main (boundary form): returns (per-particle parts, total)."""
        phi = np.zeros(self.n_particles) if phi is None else phi
        total = np.zeros(1)
        _check(load().yk_energy(self.h, _ptr(sigma), _ptr(f), _ptr(phi), _ptr(total)),
               "yk_energy")
        return phi, float(total[0])

    def yk_repulsion(self, c0=0.01, q=3):
        """Excluded-volume repulsion (Eq. repul): returns F (Np, 2), tau, phi."""
        F = np.zeros((self.n_particles, 2))
        tau = np.zeros(self.n_particles)
        phi = np.zeros(self.n_particles)
        _check(load().yk_repulsion(self.h, float(c0), int(q), _ptr(F), _ptr(tau), _ptr(phi)),
               "yk_repulsion")
        return F, tau, phi

    def yk_stokes_apply(self, sigma, op=YK_STOKES_COMPLETED, precision=YK_FP64, out=None):
        """Stokes boundary operator on a density of 2 N values (node-major):
        YK_STOKES_TRACTION (1/2 I + K*), YK_STOKES_COMPLETED (+ W) or
        YK_STOKES_VELOCITY (S, the on-surface single layer)."""
        _f64(sigma, 2 * self.n, "sigma")
        out = np.zeros(2 * self.n) if out is None else _f64(out, 2 * self.n, "out")
        _check(load().yk_stokes_apply(self.h, int(op), _ptr(sigma), _ptr(out), int(precision)),
               "yk_stokes_apply")
        return out

    def yk_mobility(self, F, tau, want_sigma=False, allow_not_converged=False):
        """Stokes mobility problem (Section 3): velocities v (Np, 2) and angular
        velocities omega (Np,) under forces F (Np, 2) and torques tau (Np,);
        also the density sigma (2 N) when want_sigma, and the solve statistics."""
        F = np.ascontiguousarray(F, dtype=np.float64).reshape(self.n_particles, 2) \
            if isinstance(F, (list, tuple, np.ndarray)) else F
        tau = np.ascontiguousarray(tau, dtype=np.float64).reshape(self.n_particles) \
            if isinstance(tau, (list, tuple, np.ndarray)) else tau
        v = np.zeros((self.n_particles, 2))
        om = np.zeros(self.n_particles)
        sig = np.zeros(2 * self.n) if want_sigma else None
        info = yk_solve_info()
        ok = (YK_OK, YK_ERR_NOT_CONVERGED) if allow_not_converged else (YK_OK,)
        rc = _check(load().yk_mobility(self.h, _ptr(F), _ptr(tau), _ptr(v), _ptr(om), _ptr(sig),
                                       C.byref(info)), "yk_mobility", ok)
        d = info.as_dict()
        d["converged"] = rc == YK_OK
        return v, om, sig, d

    def yk_step(self, n_steps=1, **kw):
        """Particle dynamics (Algorithm 1): constant drag (Eq. euler) or, with
        mobility=1, the Stokes mobility velocities (Eq. mob_vec). Returns the
        particles after n_steps (Np x 6 like the input), the energy and the
        solve statistics of every step."""
        d = default_dynamics(**kw)
        parts = (yk_particle * self.n_particles)()
        energy = np.zeros(max(n_steps, 1))
        infos = (yk_solve_info * max(n_steps, 1))()
        _check(load().yk_step(self.h, C.byref(d), int(n_steps), C.cast(parts, C.c_void_p),
                              _ptr(energy), C.cast(infos, C.c_void_p)), "yk_step")
        out = np.array([[p.shape, p.cx, p.cy, p.phi, p.A, p.B] for p in parts])
        return out, energy[:n_steps], [infos[k].as_dict() for k in range(n_steps)]

    def yk_eval_potential_near(self, sigma, targets, out=None):
        """Potential at targets anywhere in the water, also next to a boundary
        (QBX near the boundary); NaN inside particles."""
        t = np.ascontiguousarray(targets, dtype=np.float64) if isinstance(targets, (list, np.ndarray)) else targets
        nt = t.shape[0]
        u = np.zeros(nt) if out is None else out
        _check(load().yk_eval_potential_near(self.h, _ptr(sigma), _ptr(t), C.c_int64(nt), _ptr(u)),
               "yk_eval_potential_near")
        return u

    def yk_eval_potential(self, sigma, targets, out=None):
        t = np.ascontiguousarray(targets, dtype=np.float64) if isinstance(targets, (list, np.ndarray)) else targets
        nt = t.shape[0]
        out = np.zeros(nt) if out is None else out
        _check(load().yk_eval_potential(self.h, _ptr(sigma), _ptr(t), C.c_int64(nt), _ptr(out)),
               "yk_eval_potential")
        return out

    def yk_eval_potential_noalloc(self, sigma, targets, out):
        """Allocation-free potential: sigma, targets (nt x 2) and out must be
        CUDA tensors; the library uses its fixed scratch, not the allocator."""
        nt = targets.shape[0]
        _check(load().yk_eval_potential_noalloc(self.h, _ptr(sigma), _ptr(targets),
                                                C.c_int64(nt), _ptr(out)),
               "yk_eval_potential_noalloc")
        return out

    def yk_solve_forces(self, f, sigma=None, F=None, tau=None):
        sigma = np.zeros(self.n) if sigma is None else sigma
        F = np.zeros((self.n_particles, 2)) if F is None else F
        tau = np.zeros(self.n_particles) if tau is None else tau
        info = yk_solve_info()
        _check(load().yk_solve_forces(self.h, _ptr(f), _ptr(sigma), _ptr(F), _ptr(tau),
                                      C.byref(info)), "yk_solve_forces",
               (YK_OK, YK_ERR_NOT_CONVERGED))
        return sigma, F, tau, info.as_dict()


def yk_kernel_launches():
    c = C.c_uint64()
    _check(load().yk_kernel_launches(C.byref(c)), "yk_kernel_launches")
    return c.value


def yk_solve_batch(geoms, fs, sigmas=None, allow_not_converged=False):
    """Solve several configurations together (lock-step inner GMRES); geoms
    is a list of Geometry of one context, fs their data (arrays or tensors).
    Returns (sigmas, infos)."""
    n = len(geoms)
    if len(fs) != n:
        raise ValueError("one f per geometry")
    sigmas = [np.zeros(g.n) for g in geoms] if sigmas is None else sigmas
    for g, f, s in zip(geoms, fs, sigmas):
        _f64(f, g.n, "f")
        _f64(s, g.n, "sigma")
    G = (C.c_void_p * n)(*[g.h.value if hasattr(g.h, "value") else g.h for g in geoms])
    F = (C.c_void_p * n)(*[_ptr(f) for f in fs])
    S = (C.c_void_p * n)(*[_ptr(s) for s in sigmas])
    infos = (yk_solve_info * n)()
    ok = (YK_OK, YK_ERR_NOT_CONVERGED) if allow_not_converged else (YK_OK,)
    _check(load().yk_solve_batch(G, n, F, S, C.cast(infos, C.c_void_p)), "yk_solve_batch", ok)
    return sigmas, [infos[k].as_dict() for k in range(n)]


def yk_fp32_fma_peak(device=0):
    """Measured FP32 FMA throughput of the device in TFLOP/s."""
    t = C.c_double()
    _check(load().yk_fp32_fma_peak(int(device), C.byref(t)), "yk_fp32_fma_peak")
    return t.value


def default_dynamics(**kw):
    """yk_dynamics with the library defaults, overridden by keyword."""
    d = yk_dynamics()
    _check(load().yk_default_dynamics(C.byref(d)), "yk_default_dynamics")
    for k, v in kw.items():
        if not hasattr(d, k):
            raise AttributeError(k)
        setattr(d, k, v)
    return d


def params_for(workload, **kw):
    """yk_params for a named workload (paper_1810_04131_gb300.workloads)."""
    p = default_params(rho=workload.rho, n_panels=workload.n_panels, n_gl=workload.n_gl,
                       qbx_order=workload.qbx_order, gmres_tol=workload.gmres_tol)
    for k, v in kw.items():
        setattr(p, k, v)
    return p
