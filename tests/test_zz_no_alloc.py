"""The allocation-free potential entry point (yk_eval_potential_noalloc).

It is for callers that must not allocate device memory where they evaluate
the potential: real-time loops that cannot block in the allocator, or
applications that reserved the GPU's memory up front and hand the library a
fixed budget. It keeps its partial sums in a fixed device array inside the
library rather than allocating them.

Checked here, through the C ABI: on two calls in a row with different
densities, it returns what yk_eval_potential returns for the same inputs
(within the 1e-12 FP64 bar of the other parity tests). Both calls share the
fixed array, so the second one shows that stale contents from the first do
not leak into the result. Oversized requests and host pointers are
refused. This file is collected last, and it also passes when run alone in a
fresh process.
"""
import numpy as np
import pytest

from paper_1810_04131_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_potential_matches_allocating_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_04131_gb300 import yk
    wl = W.disks8()
    ctx = yk.Context(0, torch.cuda.current_stream().cuda_stream)
    g = yk.Geometry(ctx, wl.particles, yk.params_for(wl, precision=yk.YK_FP64))
    dev = torch.device("cuda", 0)
    tgt = torch.from_numpy(np.ascontiguousarray(wl.targets)).to(dev)
    rng = np.random.default_rng(17)
    for call in range(2):   # two calls in a row share the fixed scratch
        sig = torch.from_numpy(rng.standard_normal(g.n)).to(dev)
        u_ref = torch.zeros(tgt.shape[0], dtype=torch.float64, device=dev)
        g.yk_eval_potential(sig, tgt, out=u_ref)
        u = torch.full_like(u_ref, float("nan"))
        g.yk_eval_potential_noalloc(sig, tgt, u)
        torch.cuda.synchronize()
        a, b = u.cpu().numpy(), u_ref.cpu().numpy()
        assert np.isfinite(a).all(), call
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b), call

    # requests beyond the fixed scratch are refused with a clear code
    big = torch.zeros(((1 << 20) + 1, 2), dtype=torch.float64, device=dev)
    out = torch.zeros((1 << 20) + 1, dtype=torch.float64, device=dev)
    sig = torch.zeros(g.n, dtype=torch.float64, device=dev)
    with pytest.raises(yk.YKError) as e:
        g.yk_eval_potential_noalloc(sig, big, out)
    assert e.value.code == yk.YK_ERR_TOO_LARGE
    # host arrays would need staging allocations: refused
    with pytest.raises(yk.YKError) as e:
        g.yk_eval_potential_noalloc(np.zeros(g.n), np.asarray(wl.targets), np.zeros(len(wl.targets)))
    assert e.value.code == yk.YK_ERR_ARG
    g.close()
    ctx.close()
