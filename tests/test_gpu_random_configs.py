"""Seeded random configurations: the FP64 path against the restatement of Algorithm 1 plus the
direct real-space and self terms, element by element, and the mixed path against FP64.

Each case draws N, the box (free side L, periodic L3), P (even and odd), M, the padded sizes and
the upsampling split, and rc, so that tile, bin and cell boundaries, ragged tails, class splits
(n_l = 0, some, all modes) and cell stencils vary well beyond the fixed parity cases."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import direct  # noqa: E402
from oracle import se1p_algorithm as se  # noqa: E402
from paper_1611_09538_gb300 import build as se1p_build  # noqa: E402
from paper_1611_09538_gb300 import inputs, se1p  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    se1p_build.build()
    se1p.load()
    direct.build()


def smooth_at_least(n):
    while True:
        m = n
        for r in (2, 3, 5, 7):
            while m % r == 0:
                m //= r
        if m == 1:
            return n
        n += 1


def draw(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(20, 400))
    L = float(rng.choice([1.0, 1.5, 2.0]))
    L3 = float(L * rng.choice([0.5, 1.0, 1.7, 3.0]))
    P = int(rng.integers(6, 25))
    M = int(smooth_at_least(int(rng.integers(max(P, 12), 40))))
    M3 = int(smooth_at_least(max(P, int(round(M * L3 / L)))))
    Mt = smooth_at_least(M + P + int(rng.integers(0, 5)))
    n0 = smooth_at_least(int(np.ceil(2.83 * Mt)))
    nI = smooth_at_least(int(np.ceil(float(rng.uniform(1.0, 3.0)) * Mt)))
    nl = int(rng.choice([0, 1, 3, M3]))
    xi = float(rng.uniform(4.0, 9.0)) * M / 32.0 / L
    rc = float(min(L3, rng.uniform(0.15, 0.4) * L))
    x, q = inputs.uniform_shifted(n, (L, L, L3), seed=2000 + seed)
    return x, q, dict(L=(L, L, L3), xi=xi, M=(M, M, M3), P=P, Mt=Mt, n0=n0, nI=nI, nl=nl, rc=rc)


@pytest.mark.parametrize("seed", range(12))
def test_random_configuration(seed):
    x, q, prm = draw(seed)
    L = prm["L"]
    phiF, FF = se.se1p_fourier(x, q, L, prm["xi"], prm["M"], prm["P"], prm["Mt"], prm["n0"], prm["nI"], prm["nl"])
    pp, ff = direct.ewald1p_parts(x, q, L[2], prm["xi"], prm["rc"], kcut=1e300)
    phi_ref, F_ref = phiF + pp[:, 0] + pp[:, 3], FF + ff[:, 0]
    out = {}
    for prec in (se1p.SE1P_FP64, se1p.SE1P_MIXED):
        plan = se1p.Plan(L, prm["xi"], prm["M"], prm["P"], len(q), Mt=prm["Mt"], n0=prm["n0"], nI=prm["nI"],
                         nl=prm["nl"], rc=prm["rc"], precision=prec)
        r = plan.eval(torch.as_tensor(x, device="cuda"), torch.as_tensor(q, device="cuda"))
        out[prec] = (r.phi.cpu().numpy(), r.force.cpu().numpy())
        plan.close()
    phi, F = out[se1p.SE1P_FP64]
    # FP64: same finite sums in another order; the symbol may amplify rounding where eta > 1
    assert np.max(np.abs(phi - phi_ref)) < 1e-9 * np.max(np.abs(phi_ref)), prm
    assert np.max(np.abs(F - F_ref)) < 1e-9 * np.max(np.abs(F_ref)), prm
    rel = lambda a, b: np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))
    eta = prm["P"] * prm["xi"] ** 2 * (L[0] / prm["M"][0]) ** 2 / (0.95 ** 2 * np.pi)
    if eta < 1.0:  # otherwise FP32 rounding is amplified by the growing scaling (Eq. 3.3)
        assert rel(out[se1p.SE1P_MIXED][0], phi) < 1e-5, prm
        assert rel(out[se1p.SE1P_MIXED][1], F) < 1e-5, prm
