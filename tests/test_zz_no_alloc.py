"""The allocation-free real-space entry point (se1p_real_space_noalloc).

Callers that cannot allocate device memory (a framework owns the allocator,
memory is handed out up front, or allocation is forbidden after start-up) use
this variant; it keeps its scratch in a static device array.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1611_09538_gb300 import build as se1p_build  # noqa: E402
from paper_1611_09538_gb300 import inputs, se1p  # noqa: E402


def max_rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))


def _existing(params_kw, x, q):
    """phi^R, F^R from the plan-based entry point se1p_real_space."""
    n = len(q)
    plan = se1p.Plan(n_max=n, **params_kw)
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    se1p.se1p_real_space(plan.handle, n, x, q, phi, F)
    assert se1p.se1p_plan_sync_status(plan.handle) == 0
    out = phi.cpu().numpy(), F.cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("precision,tol", [(se1p.SE1P_FP64, 1e-12), (se1p.SE1P_MIXED, 1e-6)])
def test_noalloc_matches_plan_entry_point_twice(precision, tol):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    se1p_build.build()
    systems = [inputs.uniform_alternating(1200, (1.0, 1.0, 1.0), seed=31),
               inputs.uniform_shifted(777, (1.0, 1.0, 1.4), seed=32)]
    for (xn, qn), L in zip(systems, [(1.0, 1.0, 1.0), (1.0, 1.0, 1.4)]):
        kw = dict(L=L, xi=8.0, M=(32, 32, 32), P=16, rc=0.3, precision=precision)
        x = torch.as_tensor(xn, device="cuda")
        q = torch.as_tensor(qn, device="cuda")
        phi_ref, F_ref = _existing(kw, x, q)
        prm = se1p.make_params(**kw)
        n = len(qn)
        phi = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        F = torch.full((n, 3), np.nan, dtype=torch.float64, device="cuda")
        se1p.se1p_real_space_noalloc(prm, n, x, q, phi, F)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        se1p.se1p_real_space_noalloc(prm, n, x, q, phi, F)  # second call in a row, same buffers
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        assert max_rel(phi.cpu().numpy(), phi_ref) < tol
        assert max_rel(F.cpu().numpy(), F_ref) < tol


def test_noalloc_rejects_oversized_input():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    se1p_build.build()
    prm = se1p.make_params((1.0, 1.0, 1.0), 8.0, (32, 32, 32), 16, rc=0.3)
    x = torch.zeros((16385, 3), dtype=torch.float64, device="cuda")
    q = torch.zeros(16385, dtype=torch.float64, device="cuda")
    with pytest.raises(se1p.SE1PError) as ei:
        se1p.se1p_real_space_noalloc(prm, 16385, x, q, x[:, 0].contiguous(), x)
    assert ei.value.code == 8
