"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every entry point that include/yk.h declares, the ctypes
structures match the C layout, and calls fail cleanly without a device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1810_04131_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "yk.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1810_04131_gb300 import build, yk
    if not os.path.exists(yk.LIB_PATH):
        build.build()
    return yk.load()


def header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(yk_\w+)\s*\(", txt, flags=re.M)))


def test_exports_match_header(lib):
    from paper_1810_04131_gb300 import yk
    names = header_functions()
    assert len(names) >= 17
    assert sorted(yk.EXPORTS) == names
    out = subprocess.run(["nm", "-D", "--defined-only", yk.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (yk_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_struct_layout_matches_c(tmp_path):
    """sizeof/offsetof of the public structs, compiled by gcc from the header."""
    from paper_1810_04131_gb300 import yk
    src = tmp_path / "lay.c"
    fields = {
        "yk_particle": [f for f, _ in yk.yk_particle._fields_],
        "yk_params": [f for f, _ in yk.yk_params._fields_],
        "yk_solve_info": [f for f, _ in yk.yk_solve_info._fields_],
        "yk_dynamics": [f for f, _ in yk.yk_dynamics._fields_],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "yk.h"', "int main(void){"]
    for s, fs in fields.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (s, s))
        for f in fs:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (s, f, s, f))
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for s, fs in fields.items():
        cls = getattr(yk, s)
        assert int(got[s]) == C.sizeof(cls), s
        for f in fs:
            assert int(got["%s.%s" % (s, f)]) == getattr(cls, f).offset, (s, f)


def test_defaults_and_errors_without_gpu(lib):
    from paper_1810_04131_gb300 import yk
    p = yk.default_params()
    assert p.n_panels == 16 and p.n_gl == 16 and p.qbx_order == 10
    assert p.qbx_r_factor == 0.125 and p.oversample == 8 and p.near_width == 1
    assert p.precision == yk.YK_MIXED and p.gmres_tol == 1e-12
    assert p.farfield == yk.YK_FARFIELD_DENSE and p.fmm_order == 12 and p.fmm_leaf == 0.0
    assert p.coarse == yk.YK_COARSE_MODES
    assert lib.yk_default_params(None) == yk.YK_ERR_ARG
    assert lib.yk_strerror(yk.YK_ERR_BAD_GEOMETRY) == b"particles overlap"
    assert lib.yk_create(None, 0, None) == yk.YK_ERR_ARG
    assert lib.yk_destroy(None) == yk.YK_ERR_ARG
    assert lib.yk_drain(None) == yk.YK_ERR_ARG
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        h = C.c_void_p()
        rc = lib.yk_create(C.byref(h), 0, None)
        assert rc in (yk.YK_ERR_CUDA, yk.YK_ERR_ARG)
        assert not h.value


def test_workloads_are_seeded_and_separated():
    a = W.disks8()
    b = W.disks8()
    assert np.array_equal(a.particles, b.particles)
    assert np.array_equal(a.targets, b.targets)
    p = a.particles
    d = np.hypot(p[:, None, 1] - p[None, :, 1], p[:, None, 2] - p[None, :, 2])
    d[np.arange(len(p)), np.arange(len(p))] = np.inf
    assert (d - 2.0).min() >= 0.5
    assert a.n_nodes == 2048
    e = W.make_particles(30, 30.0, 0.2, seed=9, shape=W.SHAPE_ELLIPSE, A=1.0, B=0.5)
    # boundary distance by 2048 samples of each ellipse (the placement samples
    # 4096 x 1024; both stay within a few 1e-3 of the true distance)
    t = np.linspace(0.0, 2.0 * np.pi, 2048, endpoint=False)
    pts = []
    for row in e:
        c, s_ = np.cos(row[3]), np.sin(row[3])
        u, v = row[4] * np.cos(t), row[5] * np.sin(t)
        pts.append(np.stack([row[1] + c * u - s_ * v, row[2] + s_ * u + c * v], 1))
    for i in range(len(e)):
        for j in range(i):
            if np.hypot(*(e[i, 1:3] - e[j, 1:3])) > 2.0 + 0.2 + 1.0:
                continue
            dmin = np.sqrt(((pts[i][:, None] - pts[j][None]) ** 2).sum(-1)).min()
            assert dmin >= 0.2 - 5e-3, (i, j, dmin)
    s = W.request_stream(50, seed=6)
    assert len(s) == 50 and all(4 <= r["n_particles"] <= 2048 for r in s)
    assert all(8 <= r["n_panels"] <= 32 for r in s)


def test_table2_collections_as_printed():
    """Table 2: 250 / 500 / 1000 / 2000 unit disks in 100 / 200 / 200 / 400
    square boxes, N_bdy = 70 boundary points each, tolerance 1e-5; seeded,
    inside the box and at least 0.5 apart (centre distance >= 2.5)."""
    for n, box in ((250, 100.0), (500, 200.0), (1000, 200.0), (2000, 400.0)):
        wl = W.table2(n)
        assert wl.n_particles == n and wl.box == box and wl.n_panels * wl.n_gl == 70
        assert wl.n_nodes == 70 * n and wl.rho == 4.0 and wl.gmres_tol == 1e-5
        assert np.array_equal(wl.particles, W.table2(n).particles)
        c = wl.particles[:, 1:3]
        assert (c >= 1.0).all() and (c <= box - 1.0).all()
        d = np.hypot(c[:, None, 0] - c[None, :, 0], c[:, None, 1] - c[None, :, 1])
        d[np.arange(n), np.arange(n)] = np.inf
        assert d.min() >= 2.5
