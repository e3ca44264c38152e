"""Reverse-mode derivatives (systems form 3): torch.autograd over the C ABI.

* energy: dU/dx = -F and dU/dq = phi, checked against central finite differences
  of U (FP64, h = 1e-5) and against the direct oracle's forces;
* potential: the adjoint (se1p_eval_vjp) for l = sum c phi, checked against
  central finite differences in x and along neutral charge changes;
* clustered charges (Gaussian blobs, sigma = 0.05, 8 centres, L = [1,1,2]) in FP64
  and mixed precision against the oracle's analytic forces at sampled targets.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import direct  # noqa: E402
from paper_1611_09538_gb300 import build as se1p_build  # noqa: E402
from paper_1611_09538_gb300 import inputs, se1p  # noqa: E402
from paper_1611_09538_gb300.autograd import se1p_energy, se1p_potential  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    se1p_build.build()


def plan_for(n, precision=se1p.SE1P_FP64, L=(1.0, 1.0, 1.0)):
    return se1p.Plan(L, 8.0, (40, 40, 40 if L[2] == 1.0 else 80), 24, n, Mt=64, n0=192, nI=256, nl=6, rc=0.3,
                     precision=precision)


def system(n=200, seed=51):
    x, q = inputs.uniform_shifted(n, seed=seed)
    return torch.as_tensor(x, device="cuda"), torch.as_tensor(q, device="cuda")


def test_energy_gradient_is_force_and_potential():
    x, q = system()
    plan = plan_for(len(q))
    xr = x.clone().requires_grad_(True)
    qr = q.clone().requires_grad_(True)
    U = se1p_energy(plan, xr, qr)
    U.backward()
    r = plan.eval(x, q)
    # a second evaluation differs from the first only in summation order (atomics)
    assert torch.allclose(xr.grad, -r.force, rtol=0, atol=1e-12 * r.force.abs().max().item())
    assert torch.allclose(qr.grad, r.phi, rtol=0, atol=1e-12 * r.phi.abs().max().item())


def test_energy_gradient_by_finite_differences():
    x, q = system()
    plan = plan_for(len(q))
    U0 = lambda xx, qq: plan.eval(xx, qq).energy.item()
    r = plan.eval(x, q)
    h = 1e-5
    for i in (3, 50, 177):
        for d in range(3):
            xp, xm = x.clone(), x.clone()
            xp[i, d] += h
            xm[i, d] -= h
            fd = (U0(xp, q) - U0(xm, q)) / (2 * h)
            assert -fd == pytest.approx(r.force[i, d].item(), rel=1e-6, abs=1e-6 * r.force.abs().max().item())
    # neutral charge change: +h on i, -h on j
    for i, j in ((0, 1), (10, 99)):
        qp, qm = q.clone(), q.clone()
        qp[i] += h
        qp[j] -= h
        qm[i] -= h
        qm[j] += h
        fd = (U0(x, qp) - U0(x, qm)) / (2 * h)
        assert fd == pytest.approx((r.phi[i] - r.phi[j]).item(), rel=1e-6, abs=1e-8)


def test_potential_vjp_by_finite_differences():
    x, q = system(seed=52)
    n = len(q)
    plan = plan_for(n)
    c = torch.as_tensor(np.random.default_rng(3).standard_normal(n), device="cuda")
    xr = x.clone().requires_grad_(True)
    qr = q.clone().requires_grad_(True)
    loss = (c * se1p_potential(plan, xr, qr)).sum()
    loss.backward()
    L = lambda xx, qq: float((c * plan.eval(xx, qq).phi).sum())
    h = 1e-5
    gmax = xr.grad.abs().max().item()
    for i in (7, 120):
        for d in range(3):
            xp, xm = x.clone(), x.clone()
            xp[i, d] += h
            xm[i, d] -= h
            fd = (L(xp, q) - L(xm, q)) / (2 * h)
            assert xr.grad[i, d].item() == pytest.approx(fd, rel=1e-6, abs=2e-7 * gmax)
    for i, j in ((5, 6), (40, 160)):
        qp, qm = q.clone(), q.clone()
        qp[i] += h
        qp[j] -= h
        qm[i] -= h
        qm[j] += h
        fd = (L(x, qp) - L(x, qm)) / (2 * h)
        assert (qr.grad[i] - qr.grad[j]).item() == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_mixed_vjp_matches_fp64():
    x, q = system(seed=53)
    n = len(q)
    v = torch.as_tensor(np.random.default_rng(4).standard_normal(n), device="cuda")
    out = {}
    for prec in (se1p.SE1P_FP64, se1p.SE1P_MIXED):
        plan = plan_for(n, prec)
        gx = torch.empty_like(x)
        gq = torch.empty_like(q)
        se1p.se1p_eval_vjp(plan.handle, n, x, q, v, gx, gq)
        assert se1p.se1p_plan_sync_status(plan.handle) == 0
        out[prec] = (gx.cpu().numpy(), gq.cpu().numpy() - gq.cpu().numpy().mean())
    rel = lambda a, b: np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))
    assert rel(out[1][0], out[0][0]) < 1e-6
    assert rel(out[1][1], out[0][1]) < 1e-6


@pytest.mark.parametrize("precision,tol", [(se1p.SE1P_FP64, 1e-6), (se1p.SE1P_MIXED, 2e-6)])
def test_clustered_forces_match_oracle(precision, tol):
    """Gaussian blobs (the clustered differentiation workload at N = 20 000): forces
    = -dU/dx from autograd against the direct sums at sampled targets."""
    xn, qn = inputs.clustered(20000, seed=3)
    L = (1.0, 1.0, 2.0)
    x = torch.as_tensor(xn, device="cuda")
    q = torch.as_tensor(qn, device="cuda")
    plan = se1p.Plan(L, 20.0, (64, 64, 128), 24, len(qn), Mt=96, n0=288, nI=384, nl=4, rc=0.15,
                     precision=precision)
    xr = x.clone().requires_grad_(True)
    U = se1p_energy(plan, xr, q)
    U.backward()
    F = (-xr.grad).cpu().numpy()
    t = np.random.default_rng(9).choice(len(qn), 6, replace=False)
    _, F_ref, _ = direct.ewald1p(xn, qn, L[2], 20.0, 0.15, targets=t)
    rel = np.sqrt(np.sum((F[t] - F_ref) ** 2) / np.sum(F_ref ** 2))
    assert rel < tol
