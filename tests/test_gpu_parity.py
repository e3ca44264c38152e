"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Stage tests compare one step at a time with the numpy restatement of
Algorithms 1-3 (element by element, rounding-level tolerance); end-to-end
tests compare phi, F and U with the direct Ewald1P sums.

Tolerances:
  * FP64 stage parity: the GPU and the oracle evaluate the same finite sums in
    different orders (Stockham vs pocketfft FFTs, tile vs bincount sums), so
    results agree to a few hundred ulps of the largest value:
    max |diff| <= 1e-11 max |ref|.
  * FP64 end to end vs the direct sums at the parity configuration: relative
    rms <= 1e-10 (the method's own error there is ~1e-13).
  * mixed FP32/FP64 vs FP64 GPU: relative rms <= 1e-6.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import direct, se1p_algorithm as se  # noqa: E402
from paper_1611_09538_gb300 import build as se1p_build  # noqa: E402
from paper_1611_09538_gb300 import inputs, se1p  # noqa: E402


def rel_rms(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def max_rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    se1p_build.build()
    se1p.load()
    direct.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def make_plan(prm, n_max, precision=se1p.SE1P_FP64, rc=None):
    L = prm["L"]
    return se1p.Plan(L, prm["xi"], prm["M"], prm["P"], n_max, Mt=prm["Mt"], n0=prm["n0"], nI=prm["nI"],
                     nl=prm["nl"], rc=(prm.get("rc", 0.0) if rc is None else rc), precision=precision)


def small_case(n=700, L=(1.0, 1.0, 1.0), seed=3, xi=8.0, M=(40, 40, 40), P=24, Mt=64, n0=192, nI=256, nl=6,
               rc=0.3):
    x, q = inputs.uniform_alternating(n, L, seed=seed)
    return x, q, dict(L=L, xi=xi, M=M, P=P, Mt=Mt, n0=n0, nI=nI, nl=nl, rc=rc)


CASES = {
    # cubic, even P, tiles of 8 divide every axis
    "cubic_P24": small_case(),
    # ragged tiles (M3 = 30, Mt = 42), odd P, non-cubic box with its own z spacing
    "ragged_oddP": small_case(n=333, L=(1.0, 1.0, 1.3), seed=4, xi=7.0, M=(24, 24, 30), P=21, Mt=49, n0=140,
                              nI=98, nl=2, rc=0.25),
    # C1-like: P = 16, M = 32, Mt = 48
    "c1_like": small_case(n=1000, seed=0, xi=8.0, M=(32, 32, 32), P=16, Mt=48, n0=144, nI=144, nl=3),
    # plain upsampled FFT (Section 3.2: s_l = s0, n_l = k_inf): every k3 mode padded to nI = n0
    "plain_upsampled": small_case(n=500, seed=7, xi=8.0, M=(32, 32, 32), P=16, Mt=48, n0=144, nI=144, nl=16),
    # elongated periodic axis: M3 = 256 (K3 = 129 z modes, 32 of them in the set I)
    "elongated": small_case(n=600, L=(1.0, 1.0, 8.0), seed=6, xi=8.0, M=(32, 32, 256), P=16, Mt=48, n0=144,
                            nI=96, nl=4, rc=0.3),
    # short periodic axis: M3 = 16 < P + 8, so a window wraps into the same 8-point gridding tile
    "short_axis": small_case(n=400, L=(1.0, 1.0, 0.5), seed=8, xi=8.0, M=(32, 32, 16), P=16, Mt=48, n0=144,
                             nI=96, nl=2, rc=0.25),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_spread_matches_oracle(case):
    x, q, prm = CASES[case]
    g = se.Grid(prm["L"], prm["xi"], prm["M"], prm["P"], prm["Mt"], prm["n0"], prm["nI"], prm["nl"])
    H_ref = se.spread(g, x, q)
    plan = make_plan(prm, len(q))
    grid = torch.zeros(plan.grid_shape(), dtype=torch.float64, device="cuda")
    se1p.se1p_spread(plan.handle, len(q), dev(x), dev(q), grid)
    torch.cuda.synchronize()
    assert max_rel(grid.cpu().numpy(), H_ref) < 1e-12


@pytest.mark.parametrize("case", sorted(CASES))
def test_fourier_matches_oracle(case):
    x, q, prm = CASES[case]
    g = se.Grid(prm["L"], prm["xi"], prm["M"], prm["P"], prm["Mt"], prm["n0"], prm["nI"], prm["nl"])
    H = se.spread(g, x, q)
    Ht_ref = se.fourier_solve(g, H)
    plan = make_plan(prm, len(q))
    out = torch.zeros_like(dev(H))
    se1p.se1p_fourier(plan.handle, dev(H), out)
    torch.cuda.synchronize()
    assert max_rel(out.cpu().numpy(), Ht_ref) < 1e-11


@pytest.mark.parametrize("case", sorted(CASES))
def test_gather_matches_oracle(case):
    x, q, prm = CASES[case]
    g = se.Grid(prm["L"], prm["xi"], prm["M"], prm["P"], prm["Mt"], prm["n0"], prm["nI"], prm["nl"])
    Ht = se.fourier_solve(g, se.spread(g, x, q))
    phi_ref, F_ref = se.gather(g, Ht, x, q)
    plan = make_plan(prm, len(q))
    phi = torch.empty(len(q), dtype=torch.float64, device="cuda")
    F = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
    se1p.se1p_gather(plan.handle, len(q), dev(x), dev(q), dev(Ht), phi, F)
    torch.cuda.synchronize()
    assert max_rel(phi.cpu().numpy(), phi_ref) < 1e-12
    assert max_rel(F.cpu().numpy(), F_ref) < 1e-12


def test_gather_long_list_matches_oracle():
    """A particle list long enough for the gather's per-SM handout (at least 16 particles per resident
    warp: 77 824 on 152 SMs in mixed precision, fewer in FP64), with a ragged tail, against Step 6 of
    the oracle on one random grid, every particle; a second gather on twice the grid (the handout's
    cursors start again from zero) gives twice the values.  Tolerances: FP64 as the stage tests; mixed
    rounds the grid to FP32 and sums in FP32, relative rms <= 1e-6 and max |diff| <= 1e-5 max |ref|."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 20 * 32 * sms + 37
    x, q = inputs.uniform_alternating(n, seed=12)
    prm = dict(L=(1.0, 1.0, 1.0), xi=8.0, M=(32, 32, 32), P=16, Mt=48, n0=144, nI=144, nl=3, rc=0.15)
    g = se.Grid(prm["L"], prm["xi"], prm["M"], prm["P"], prm["Mt"], prm["n0"], prm["nI"], prm["nl"])
    Ht = np.random.default_rng(13).standard_normal((prm["M"][2], prm["Mt"], prm["Mt"]))
    phi_ref, F_ref = se.gather(g, Ht, x, q)
    for precision, tol_rms, tol_max in ((se1p.SE1P_FP64, 1e-12, 1e-12), (se1p.SE1P_MIXED, 1e-6, 1e-5)):
        plan = make_plan(prm, n, precision=precision)
        for scale in (1.0, 2.0):
            phi = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            F = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
            se1p.se1p_gather(plan.handle, n, dev(x), dev(q), dev(scale * Ht), phi, F)
            torch.cuda.synchronize()
            assert se1p.se1p_plan_sync_status(plan.handle) == 0
            ph, ff = phi.cpu().numpy(), F.cpu().numpy()
            assert rel_rms(ph, scale * phi_ref) < tol_rms, (precision, scale)
            assert rel_rms(ff, scale * F_ref) < tol_rms, (precision, scale)
            assert max_rel(ph, scale * phi_ref) < tol_max, (precision, scale)
            assert max_rel(ff, scale * F_ref) < tol_max, (precision, scale)


@pytest.mark.parametrize("case", sorted(CASES))
def test_real_space_matches_oracle(case):
    x, q, prm = CASES[case]
    pp, ff = direct.ewald1p_parts(x, q, prm["L"][2], prm["xi"], prm["rc"])
    plan = make_plan(prm, len(q))
    phi = torch.empty(len(q), dtype=torch.float64, device="cuda")
    F = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
    se1p.se1p_real_space(plan.handle, len(q), dev(x), dev(q), phi, F)
    torch.cuda.synchronize()
    assert max_rel(phi.cpu().numpy(), pp[:, 0]) < 1e-12
    assert max_rel(F.cpu().numpy(), ff[:, 0]) < 1e-12


@pytest.mark.parametrize("case", sorted(CASES))
def test_full_eval_matches_algorithm_oracle(case):
    """se1p_eval = Algorithm 1 (numpy) + direct real space + self, element by element."""
    x, q, prm = CASES[case]
    phiF, FF = se.se1p_fourier(x, q, prm["L"], prm["xi"], prm["M"], prm["P"], prm["Mt"], prm["n0"], prm["nI"],
                               prm["nl"])
    pp, ff = direct.ewald1p_parts(x, q, prm["L"][2], prm["xi"], prm["rc"])
    phi_ref = phiF + pp[:, 0] + pp[:, 3]
    F_ref = FF + ff[:, 0]
    plan = make_plan(prm, len(q))
    r = plan.eval(dev(x), dev(q))
    phi = r.phi.cpu().numpy()
    F = r.force.cpu().numpy()
    assert max_rel(phi, phi_ref) < 1e-11
    assert max_rel(F, F_ref) < 1e-11
    U_ref = 0.5 * float(np.dot(q, phi_ref))
    assert r.energy.item() == pytest.approx(U_ref, rel=1e-11, abs=1e-11 * np.abs(q * phi_ref).sum())


def test_parity_config_matches_direct_sums():
    """P0: N=1000, xi=8, M=40^3, P=24, s_l=4, n_l=6 - GPU FP64 vs the direct Ewald1P sums <= 1e-10."""
    s = inputs.parity_p0()
    p = s.params
    phi_ref, F_ref, U_ref = direct.ewald1p(s.x, s.q, s.L[2], p["xi"], p["rc"])
    plan = make_plan(dict(p, L=s.L), len(s.q))
    r = plan.eval(dev(s.x), dev(s.q))
    assert rel_rms(r.phi.cpu().numpy(), phi_ref) < 1e-10
    assert rel_rms(r.force.cpu().numpy(), F_ref) < 1e-10
    assert r.energy.item() == pytest.approx(U_ref, rel=1e-10)


@pytest.mark.parametrize("case", ["cubic_P24", "c1_like", "plain_upsampled"])
def test_mixed_matches_fp64(case):
    x, q, prm = CASES[case]
    p64 = make_plan(prm, len(q))
    p32 = make_plan(prm, len(q), precision=se1p.SE1P_MIXED)
    r64 = p64.eval(dev(x), dev(q))
    r32 = p32.eval(dev(x), dev(q))
    assert rel_rms(r32.phi.cpu().numpy(), r64.phi.cpu().numpy()) < 1e-6
    assert rel_rms(r32.force.cpu().numpy(), r64.force.cpu().numpy()) < 1e-6
    assert r32.energy.item() == pytest.approx(r64.energy.item(), rel=1e-6)


def test_empty_system():
    x, q, prm = CASES["cubic_P24"]
    plan = make_plan(prm, 10)
    e = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    se1p.se1p_eval(plan.handle, 0, None, None, None, None, e)
    assert se1p.se1p_plan_sync_status(plan.handle) == 0
    assert e.item() == 0.0


def test_capacity_and_status_codes():
    x, q, prm = CASES["cubic_P24"]
    plan = make_plan(prm, 100)
    with pytest.raises(se1p.SE1PError) as ei:
        se1p.se1p_eval(plan.handle, 101, dev(x[:101]), dev(q[:101]))
    assert ei.value.code == 1
    # out of box in x: evaluated on clamped values, reported on sync
    xb = x[:100].copy()
    xb[5, 0] = 1.5
    phi = torch.empty(100, dtype=torch.float64, device="cuda")
    se1p.se1p_eval(plan.handle, 100, dev(xb), dev(q[:100]), phi)
    assert se1p.se1p_plan_sync_status(plan.handle) == 3
    # non-neutral
    qb = q[:100].copy()
    qb[0] += 0.5
    se1p.se1p_eval(plan.handle, 100, dev(x[:100]), dev(qb), phi)
    assert se1p.se1p_plan_sync_status(plan.handle) == 2
    # NaN
    xn = x[:100].copy()
    xn[7, 2] = np.nan
    se1p.se1p_eval(plan.handle, 100, dev(xn), dev(q[:100]), phi)
    assert se1p.se1p_plan_sync_status(plan.handle) == 7
    # status is cleared by the read
    se1p.se1p_eval(plan.handle, 100, dev(x[:100]), dev(q[:100]), phi)
    assert se1p.se1p_plan_sync_status(plan.handle) == 0


def test_z_wrapping_and_host_entry_point():
    x, q, prm = CASES["cubic_P24"]
    plan = make_plan(prm, len(q))
    r = plan.eval(dev(x), dev(q))
    xs = x.copy()
    xs[:, 2] += 3.0  # three periods up
    phi = np.empty(len(q))
    F = np.empty((len(q), 3))
    en = np.empty(1)
    se1p.se1p_eval_host(plan.handle, len(q), np.ascontiguousarray(xs), np.ascontiguousarray(q), phi, F, en)
    assert max_rel(phi, r.phi.cpu().numpy()) < 1e-12
    assert max_rel(F, r.force.cpu().numpy()) < 1e-11


@pytest.mark.parametrize("precision", [se1p.SE1P_FP64, se1p.SE1P_MIXED])
def test_back_to_back_evaluations_on_one_plan(precision):
    """Consecutive evaluations with different charges on one plan, queued without a host sync:
    the real space runs on the plan's second stream (fork after the pack, join before the
    finalisation), so each result must equal that of a fresh plan, element by element."""
    x, q0, prm = CASES["c1_like"]
    qs = [q0, q0[::-1].copy(), np.roll(q0, 7)]
    plan = make_plan(prm, len(q0), precision=precision)
    xd = dev(x)
    outs = []
    for qq in qs:
        phi = torch.empty(len(qq), dtype=torch.float64, device="cuda")
        F = torch.empty((len(qq), 3), dtype=torch.float64, device="cuda")
        E = torch.empty(1, dtype=torch.float64, device="cuda")
        se1p.se1p_eval(plan.handle, len(qq), xd, dev(qq), phi, F, E, torch.cuda.current_stream())
        outs.append((phi, F, E))
    torch.cuda.synchronize()
    for qq, (phi, F, E) in zip(qs, outs):
        ref = make_plan(prm, len(qq), precision=precision).eval(xd, dev(qq))
        tol = 1e-12 if precision == se1p.SE1P_FP64 else 1e-6  # atomics: summation order only
        assert max_rel(phi.cpu().numpy(), ref.phi.cpu().numpy()) < tol
        assert max_rel(F.cpu().numpy(), ref.force.cpu().numpy()) < tol
        assert E.item() == pytest.approx(ref.energy.item(), rel=tol)


@pytest.mark.parametrize("precision", [se1p.SE1P_FP64, se1p.SE1P_MIXED])
def test_profiling_modes_give_the_same_results(precision):
    """Profiling mode 2 runs the stages in sequence (the real space after the gather, adding into
    the same outputs) instead of overlapping them: the results equal the overlapped evaluation's up
    to the order of the atomic additions, and every stage is recorded."""
    x, q, prm = CASES["cubic_P24"]
    plan = make_plan(prm, len(q), precision=precision)
    xd, qd = dev(x), dev(q)
    ref = plan.eval(xd, qd)
    tol = 1e-12 if precision == se1p.SE1P_FP64 else 1e-6
    for mode in (1, 2):
        se1p.se1p_plan_set_profiling(plan.handle, mode)
        r = plan.eval(xd, qd)
        ms, ne = se1p.se1p_plan_stage_times(plan.handle)
        assert ne == 1 and all(v > 0 for v in ms.values())
        assert max_rel(r.phi.cpu().numpy(), ref.phi.cpu().numpy()) < tol
        assert max_rel(r.force.cpu().numpy(), ref.force.cpu().numpy()) < tol
        assert r.energy.item() == pytest.approx(ref.energy.item(), rel=tol)
    se1p.se1p_plan_set_profiling(plan.handle, 0)
    with pytest.raises(se1p.SE1PError):
        se1p.se1p_plan_set_profiling(plan.handle, 3)
    plan.close()
