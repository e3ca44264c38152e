"""The triply periodic Spectral Ewald variant (SE3P), the method the paper compares SE1P with
(Section 1, Example 6.5), against the direct triply periodic Ewald sums of the oracle.

Same gridding and gathering kernels as SE1P on the M + P extended grid, folded onto the periodic
M grid; unpadded FFTs with the Green's function 1/k^2 (no k = 0 term); real space with images in
x, y and z.  FP64 runs must reproduce the direct sums to 1e-10 at converged parameters, mixed runs
must stay within 1e-6 of FP64.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import direct  # noqa: E402
from paper_1611_09538_gb300 import build as se1p_build  # noqa: E402
from paper_1611_09538_gb300 import inputs, se1p  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
F3P = se1p.SE1P_FLAG_TRIPLY_PERIODIC


def rel_rms(a, b):
    return float(np.sqrt(np.sum((np.asarray(a) - np.asarray(b)) ** 2) / np.sum(np.asarray(b) ** 2)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    se1p_build.build()


def run(x, q, L, xi, M, P, rc, precision=se1p.SE1P_FP64):
    plan = se1p.Plan(L, xi, M, P, len(q), rc=rc, precision=precision, flags=F3P)
    r = plan.eval(torch.as_tensor(x, device="cuda"), torch.as_tensor(q, device="cuda"))
    out = r.phi.cpu().numpy(), r.force.cpu().numpy(), r.energy.item()
    plan.close()
    return out


@pytest.mark.parametrize("L,M", [((1.0, 1.0, 1.0), (40, 40, 40)), ((1.0, 1.0, 1.5), (40, 40, 60))])
def test_kspace_and_self_match_direct_sums(L, M):
    """rc <= 0: the Fourier part plus the self term, element by element, cubic and elongated."""
    x, q = inputs.uniform_alternating(400, L, seed=41)
    phi, F, _ = run(x, q, L, 8.0, M, 24, 0.0)
    pp, ff = direct.ewald3p_parts(x, q, L, 8.0, 0.0)
    assert rel_rms(phi, pp[:, 1] + pp[:, 2]) < 1e-10
    assert rel_rms(F, ff[:, 1]) < 1e-10


def test_total_matches_direct_sums_at_matched_cutoff():
    """Real space with x, y and z images within rc = 0.3 plus the Fourier and self parts."""
    L = (1.0, 1.0, 1.0)
    x, q = inputs.uniform_shifted(500, L, seed=42)
    phi, F, U = run(x, q, L, 8.0, (40, 40, 40), 24, 0.3)
    pp, ff = direct.ewald3p_parts(x, q, L, 8.0, 0.3)
    assert rel_rms(phi, pp.sum(axis=1)) < 1e-10
    assert rel_rms(F, ff.sum(axis=1)) < 1e-10
    assert abs(U - 0.5 * q @ pp.sum(axis=1)) < 1e-10 * abs(U)


def test_rock_salt_madelung_constant():
    """The eight ions of the NaCl cell (charges on grid nodes): every ion at -q M / r0, no force."""
    with open(os.path.join(GOLDEN, "madelung.json")) as f:
        m = json.load(f)["NaCl"]
    x = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                  [.5, .5, .5], [.5, 0, 0], [0, .5, 0], [0, 0, .5]], dtype=np.float64)
    q = np.array([1, 1, 1, 1, -1, -1, -1, -1], dtype=np.float64)
    phi, F, U = run(x, q, (1.0, 1.0, 1.0), 6.0, (32, 32, 32), 24, 1.0)
    np.testing.assert_allclose(phi, -q * m["M"] / m["r0"], rtol=1e-10, atol=0)
    assert np.max(np.abs(F)) < 1e-9
    assert U == pytest.approx(-8 * m["M"] / m["r0"] / 2, rel=1e-10)


def test_wrapped_positions_are_periodic_images():
    """x, y, z outside the box are wrapped: shifting charges by whole periods changes nothing."""
    L = (1.0, 1.0, 1.2)
    x, q = inputs.uniform_alternating(300, L, seed=43)
    shift = np.zeros_like(x)
    shift[::3, 0] = 1.0
    shift[1::3, 1] = -2.0
    shift[2::3, 2] = 3 * 1.2
    a = run(x, q, L, 8.0, (32, 32, 40), 16, 0.3)
    b = run(x + shift * np.array([1.0, 1.0, 1.0]), q, L, 8.0, (32, 32, 40), 16, 0.3)
    assert rel_rms(b[0], a[0]) < 1e-12 and rel_rms(b[1], a[1]) < 1e-12


def test_mixed_precision_within_1e6_of_fp64():
    """A Table 6.1 shape (N = 20 000, N/L^3 = 125, xi = 4, P = 12, rc = 0.781) on M = 54, the
    smallest 2^a 3^b 5^c 7^d size at or above the printed 52 (the FFTs run on M itself)."""
    L = (5.43, 5.43, 5.43)
    x, q = inputs.uniform_shifted(20000, L, seed=61)
    a = run(x, q, L, 4.0, (54, 54, 54), 12, 0.781, se1p.SE1P_FP64)
    b = run(x, q, L, 4.0, (54, 54, 54), 12, 0.781, se1p.SE1P_MIXED)
    assert rel_rms(b[0], a[0]) < 1e-6
    assert rel_rms(b[1], a[1]) < 1e-6
    assert abs(b[2] - a[2]) < 1e-6 * abs(a[2])

