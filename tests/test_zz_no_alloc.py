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


@pytest.mark.parametrize("precision,tol", [(se1p.SE1P_FP64, 1e-12), (se1p.SE1P_MIXED, 1e-6)])
def test_noalloc_coarsened_cell_list(precision, tol):
    """Many cells per rc-sized stencil: L = (1, 1, 7.5) at rc = 0.05 asks for 20 x 20 x 150 cells, which
    the 4096-cell cap halves to 10 x 20 x 19 (an odd count of 0.39-long cells on the periodic axis),
    so every target's sources come from merged cells several rc wide.  Same results as the plan path,
    whose cells are rc/3."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    se1p_build.build()
    L = (1.0, 1.0, 7.5)
    xn, qn = inputs.uniform_alternating(10_000, L, seed=33)
    kw = dict(L=L, xi=60.0, M=(16, 16, 120), P=8, rc=0.05, precision=precision)
    x = torch.as_tensor(xn, device="cuda")
    q = torch.as_tensor(qn, device="cuda")
    phi_ref, F_ref = _existing(kw, x, q)
    n = len(qn)
    phi = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    F = torch.full((n, 3), np.nan, dtype=torch.float64, device="cuda")
    prm = se1p.make_params(**kw)
    for _ in range(2):
        se1p.se1p_real_space_noalloc(prm, n, x, q, phi, F)
        torch.cuda.synchronize()
        assert max_rel(phi.cpu().numpy(), phi_ref) < tol
        assert max_rel(F.cpu().numpy(), F_ref) < tol


def test_noalloc_at_capacity():
    """n = 16384, the largest call the static array holds, against the plan path (FP64)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    se1p_build.build()
    xn, qn = inputs.uniform_shifted(16384, (1.0, 1.0, 1.0), seed=34)
    kw = dict(L=(1.0, 1.0, 1.0), xi=20.0, M=(32, 32, 32), P=16, rc=0.15, precision=se1p.SE1P_FP64)
    x = torch.as_tensor(xn, device="cuda")
    q = torch.as_tensor(qn, device="cuda")
    phi_ref, F_ref = _existing(kw, x, q)
    phi = torch.empty(16384, dtype=torch.float64, device="cuda")
    F = torch.empty((16384, 3), dtype=torch.float64, device="cuda")
    se1p.se1p_real_space_noalloc(se1p.make_params(**kw), 16384, x, q, phi, F)
    torch.cuda.synchronize()
    assert max_rel(phi.cpu().numpy(), phi_ref) < 1e-12
    assert max_rel(F.cpu().numpy(), F_ref) < 1e-12


def test_noalloc_matches_the_direct_real_space_sum():
    """FP64 phi^R and F^R (Eq. 2.2 and its gradient) against the oracle's direct sums over the z
    images, in a unit box and in a box whose period (0.35) is shorter than 2 rc."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import direct
    se1p_build.build()
    for L, n, seed in (((1.0, 1.0, 1.0), 500, 35), ((1.0, 1.0, 0.35), 300, 36)):
        xn, qn = inputs.uniform_alternating(n, L, seed=seed)
        rc = 0.3
        pp, ff = direct.ewald1p_parts(xn, qn, L[2], 8.0, rc)
        prm = se1p.make_params(L, 8.0, (16, 16, 16), 8, rc=rc, precision=se1p.SE1P_FP64)
        x = torch.as_tensor(xn, device="cuda")
        q = torch.as_tensor(qn, device="cuda")
        phi = torch.empty(n, dtype=torch.float64, device="cuda")
        F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        se1p.se1p_real_space_noalloc(prm, n, x, q, phi, F)
        torch.cuda.synchronize()
        assert max_rel(phi.cpu().numpy(), pp[:, 0]) < 1e-12
        assert max_rel(F.cpu().numpy(), ff[:, 0]) < 1e-12
