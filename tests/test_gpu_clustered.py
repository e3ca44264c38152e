"""The clustered workload at full size: N = 200 000 charges in 8 Gaussian blobs (sigma = 0.05)
in L = [1, 1, 2], xi = 20, M = 64 x 64 x 128, P = 24, s_l = 4, rc = 0.15.

Each charge has ~1e4 neighbours inside rc in the blobs (against ~1.3e3 in the uniform C2
workload), so the real space dominates and its atomics are heavily contended.  Checks:
  * mixed FP32/FP64 against FP64: relative rms <= 1e-6 for phi and F;
  * FP64 against the direct Ewald1P sums at sampled targets (the same parameters);
  * the energy's autograd gradient equals -F (the adjoint path at full size)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import direct  # noqa: E402
from paper_1611_09538_gb300 import build as se1p_build  # noqa: E402
from paper_1611_09538_gb300 import inputs, se1p  # noqa: E402
from paper_1611_09538_gb300.autograd import se1p_energy  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    se1p_build.build()
    se1p.load()
    direct.build()


def rel(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


@pytest.fixture(scope="module")
def c4():
    s = inputs.config_c4()
    p = s.params
    x = torch.as_tensor(s.x, device="cuda")
    q = torch.as_tensor(s.q, device="cuda")
    out = {}
    for prec in (se1p.SE1P_FP64, se1p.SE1P_MIXED):
        plan = se1p.Plan(s.L, p["xi"], p["M"], p["P"], len(s.q), Mt=p["Mt"], n0=p["n0"], nI=p["nI"],
                         nl=p["nl"], rc=p["rc"], precision=prec)
        r = plan.eval(x, q)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = plan.eval(x, q)
        torch.cuda.synchronize()
        out[prec] = (r.phi.cpu().numpy(), r.force.cpu().numpy(), r.energy.item(), time.perf_counter() - t0, plan)
    return s, x, q, out


def test_c4_mixed_vs_fp64(c4):
    s, _, _, out = c4
    phi64, F64, U64, t64, _ = out[se1p.SE1P_FP64]
    phim, Fm, Um, tm, _ = out[se1p.SE1P_MIXED]
    print(f"C4 N={len(s.q)}: FP64 {t64 * 1e3:.1f} ms, mixed {tm * 1e3:.1f} ms; mixed vs FP64 phi "
          f"{rel(phim, phi64):.2e}, F {rel(Fm, F64):.2e}, U {abs(Um - U64) / abs(U64):.2e}")
    assert rel(phim, phi64) < 1e-6
    assert rel(Fm, F64) < 1e-6


def test_c4_fp64_vs_direct_sums(c4):
    s, _, _, out = c4
    p = s.params
    phi64, F64 = out[se1p.SE1P_FP64][0], out[se1p.SE1P_FP64][1]
    t = np.random.default_rng(11).choice(len(s.q), 2, replace=False)
    phi_ref, F_ref, _ = direct.ewald1p(s.x, s.q, s.L[2], p["xi"], p["rc"], targets=t)
    print(f"C4 FP64 vs direct sums at {len(t)} targets: phi {rel(phi64[t], phi_ref):.2e}, "
          f"F {rel(F64[t], F_ref):.2e}")
    # the method's own error at these parameters (k_inf, P, s_l for ~1e-6), not rounding
    assert rel(phi64[t], phi_ref) < 1e-5
    assert rel(F64[t], F_ref) < 1e-5


def test_c4_energy_gradient_is_minus_force(c4):
    s, x, q, out = c4
    plan = out[se1p.SE1P_MIXED][4]
    xr = x.clone().requires_grad_(True)
    U = se1p_energy(plan, xr, q)
    U.backward()
    Fm = out[se1p.SE1P_MIXED][1]
    assert rel(-xr.grad.cpu().numpy(), Fm) < 1e-6
