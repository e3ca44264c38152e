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
    P = int(rng.integers(6, 25)) if seed < 100 else int(rng.integers(2, 33))  # the whole range for 100+
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


@pytest.mark.parametrize("seed", list(range(12)) + list(range(100, 106)))
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


def reference_parts(x, q, prm):
    """phi and F of Algorithm 1 plus the direct real-space and self terms."""
    L = prm["L"]
    phiF, FF = se.se1p_fourier(x, q, L, prm["xi"], prm["M"], prm["P"], prm["Mt"], prm["n0"], prm["nI"], prm["nl"])
    pp, ff = direct.ewald1p_parts(x, q, L[2], prm["xi"], prm["rc"], kcut=1e300)
    return phiF + pp[:, 0] + pp[:, 3], FF + ff[:, 0]


@pytest.mark.parametrize("seed", [0, 3, 4, 6, 8, 11])
def test_random_configuration_vjp(seed):
    """Adjoint of l = sum_i c_i phi_i.  The discrete method is a symmetric pair sum,
    phi_i = sum_j A(x_i, x_j) q_j with the same window on both sides (Eqs. 3.7, 3.11), so
    dl/dq = phi[c] (the potential of charges c) and dl/dx_k = -(c_k E_k[q] + q_k E_k[c]),
    E = F / q the field: two evaluations of the oracle at the same parameters."""
    x, q, prm = draw(seed)
    rng = np.random.default_rng(3000 + seed)
    c = rng.standard_normal(len(q))
    c -= c.mean()
    phi_q, F_q = reference_parts(x, q, prm)
    phi_c, F_c = reference_parts(x, c, prm)
    gx_ref = -(c / q)[:, None] * F_q - (q / c)[:, None] * F_c
    gq_ref = phi_c
    L = prm["L"]
    out = {}
    for prec in (se1p.SE1P_FP64, se1p.SE1P_MIXED):
        plan = se1p.Plan(L, prm["xi"], prm["M"], prm["P"], len(q), Mt=prm["Mt"], n0=prm["n0"], nI=prm["nI"],
                         nl=prm["nl"], rc=prm["rc"], precision=prec)
        xd, qd = torch.as_tensor(x, device="cuda"), torch.as_tensor(q, device="cuda")
        gx, gq = torch.empty_like(xd), torch.empty_like(qd)
        se1p.se1p_eval_vjp(plan.handle, len(q), xd, qd, torch.as_tensor(c, device="cuda"), gx, gq)
        assert se1p.se1p_plan_sync_status(plan.handle) == 0
        out[prec] = (gx.cpu().numpy(), gq.cpu().numpy())
        plan.close()
    gx, gq = out[se1p.SE1P_FP64]
    assert np.max(np.abs(gx - gx_ref)) < 1e-9 * np.max(np.abs(gx_ref)), prm
    assert np.max(np.abs(gq - gq_ref)) < 1e-9 * np.max(np.abs(gq_ref)), prm
    rel = lambda a, b: np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))
    assert rel(out[se1p.SE1P_MIXED][0], gx) < 1e-5, prm
    assert rel(out[se1p.SE1P_MIXED][1], gq) < 1e-5, prm


@pytest.mark.parametrize("P", [4, 5, 8, 9, 16])
def test_charges_on_grid_nodes(P):
    """Charges on grid nodes and half-way between them, including x = 0, y = 0 and z = 0 and
    z outside [0, L3): the grid coordinate then sits on the support-start decision (an
    integer for even P, a half-integer for odd P, Eq. 3.7's P-point support), where the two
    supports at a tie differ by the window's tail.  The FP64 path must pick the support of
    the plain definition, floor of the rounded x / h, element by element like the oracle."""
    L, M = (1.0, 1.0, 1.3), (32, 32, 40)
    h, hz = L[0] / M[0], L[2] / M[2]
    rng = np.random.default_rng(4000 + P)
    n = 300
    flat = rng.choice(2 * M[0] * 2 * M[1] * 2 * M[2], size=n, replace=False)  # unique half-node sites
    ix, rest = flat % (2 * M[0]), flat // (2 * M[0])
    iy, iz = rest % (2 * M[1]), rest // (2 * M[1])
    x = np.stack([ix * (h / 2), iy * (h / 2), iz * (hz / 2)], axis=1)
    x[:3] = [[0.0, 0.0, 0.0], [0.0, 5 * h, 7 * hz], [9 * h, 0.0, 0.0]]
    x[3:6] = [[2 * h, 3 * h, 3 * hz], [4 * h, 5 * h, 5 * hz], [6 * h, 7 * h, 9 * hz]]
    x[3:6, 2] += np.array([-1.0, 1.0, 2.0]) * L[2]  # images: wrapped in the evaluation
    q = rng.uniform(-1.0, 1.0, n)
    q -= q.mean()
    Mt = smooth_at_least(M[0] + P)
    prm = dict(L=L, xi=8.0, M=M, P=P, Mt=Mt, n0=smooth_at_least(3 * Mt), nI=smooth_at_least(2 * Mt), nl=3,
               rc=0.3)
    phi_ref, F_ref = reference_parts(x, q, prm)
    plan = se1p.Plan(L, prm["xi"], M, P, n, Mt=Mt, n0=prm["n0"], nI=prm["nI"], nl=3, rc=0.3,
                     precision=se1p.SE1P_FP64)
    r = plan.eval(torch.as_tensor(x, device="cuda"), torch.as_tensor(q, device="cuda"))
    phi, F = r.phi.cpu().numpy(), r.force.cpu().numpy()
    plan.close()
    assert np.max(np.abs(phi - phi_ref)) < 1e-10 * np.max(np.abs(phi_ref))
    assert np.max(np.abs(F - F_ref)) < 1e-10 * np.max(np.abs(F_ref))


@pytest.mark.parametrize("precision", [se1p.SE1P_FP64, se1p.SE1P_MIXED])
def test_random_configurations_in_one_batch(precision):
    """The random configurations above as one batch (one captured graph over plans that differ in
    box, P, grid, padding, class split and rc): every system's phi, F and U against the restatement
    of Algorithm 1 plus the direct real-space and self terms (FP64 element by element; mixed at the
    mixed path's tolerance, for systems with eta < 1)."""
    seeds = [0, 2, 4, 6, 9, 11, 101, 103, 104]
    cases = [draw(s) for s in seeds]
    params = [se1p.make_params(prm["L"], prm["xi"], prm["M"], prm["P"], Mt=prm["Mt"], n0=prm["n0"], nI=prm["nI"],
                               nl=prm["nl"], rc=prm["rc"], precision=precision) for _, _, prm in cases]
    ns = [len(q) for _, q, _ in cases]
    offsets = np.concatenate([[0], np.cumsum(ns)]).astype(int)
    x = torch.as_tensor(np.concatenate([c[0] for c in cases]), device="cuda").contiguous()
    q = torch.as_tensor(np.concatenate([c[1] for c in cases]), device="cuda").contiguous()
    ntot = int(offsets[-1])
    phi = torch.empty(ntot, dtype=torch.float64, device="cuda")
    F = torch.empty((ntot, 3), dtype=torch.float64, device="cuda")
    E = torch.empty(len(cases), dtype=torch.float64, device="cuda")
    b = se1p.se1p_batch_create(params, ns)
    se1p.se1p_batch_eval(b, offsets, x, q, phi, F, E)
    assert se1p.se1p_batch_sync_status(b) == 0
    se1p.se1p_batch_destroy(b)
    phi, F, E = phi.cpu().numpy(), F.cpu().numpy(), E.cpu().numpy()
    rel = lambda a, c: np.sqrt(np.sum((a - c) ** 2) / np.sum(c ** 2))
    for i, (xs, qs, prm) in enumerate(cases):
        a, c = offsets[i], offsets[i + 1]
        phi_ref, F_ref = reference_parts(xs, qs, prm)
        U_ref = 0.5 * float(qs @ phi_ref)
        if precision == se1p.SE1P_FP64:
            assert np.max(np.abs(phi[a:c] - phi_ref)) < 1e-9 * np.max(np.abs(phi_ref)), prm
            assert np.max(np.abs(F[a:c] - F_ref)) < 1e-9 * np.max(np.abs(F_ref)), prm
            assert abs(E[i] - U_ref) < 1e-9 * float(np.abs(qs) @ np.abs(phi_ref)), prm
        else:
            eta = prm["P"] * prm["xi"] ** 2 * (prm["L"][0] / prm["M"][0]) ** 2 / (0.95 ** 2 * np.pi)
            if eta < 1.0:
                assert rel(phi[a:c], phi_ref) < 1e-5, prm
                assert rel(F[a:c], F_ref) < 1e-5, prm


@pytest.mark.parametrize("M3,P", [(4, 4), (5, 5), (6, 4)])
def test_periodic_axis_shorter_than_a_tile(M3, P):
    """A periodic axis of fewer grid points than one 8-point gridding tile (M3 < 8, P up to M3): the
    tile's rows beyond M3 are never written and every window wraps around the whole axis."""
    L = (1.0, 1.0, 0.25)
    M = (16, 16, M3)
    n = 150
    x, q = inputs.uniform_shifted(n, L, seed=5000 + M3)
    Mt = smooth_at_least(M[0] + P)
    prm = dict(L=L, xi=8.0, M=M, P=P, Mt=Mt, n0=smooth_at_least(3 * Mt), nI=smooth_at_least(2 * Mt), nl=1,
               rc=0.2)
    phi_ref, F_ref = reference_parts(x, q, prm)
    for prec in (se1p.SE1P_FP64, se1p.SE1P_MIXED):
        plan = se1p.Plan(L, prm["xi"], M, P, n, Mt=Mt, n0=prm["n0"], nI=prm["nI"], nl=1, rc=0.2, precision=prec)
        r = plan.eval(torch.as_tensor(x, device="cuda"), torch.as_tensor(q, device="cuda"))
        phi, F = r.phi.cpu().numpy(), r.force.cpu().numpy()
        plan.close()
        tol = 1e-9 if prec == se1p.SE1P_FP64 else 1e-5
        assert np.max(np.abs(phi - phi_ref)) < tol * np.max(np.abs(phi_ref)), (M3, P, prec)
        assert np.max(np.abs(F - F_ref)) < tol * np.max(np.abs(F_ref)), (M3, P, prec)
