"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a library
special function, an independent quadrature, a closed form, brute-force image
sums, finite differences, invariances of the exact sum, or numbers the paper
prints.  All run on the CPU.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle import se1p_algorithm as se

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_rms(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


# ---------------------------------------------------------------- special functions (App. A)

@pytest.mark.parametrize("x", [1e-12, 1e-6, 0.01, 0.3, 0.7, 0.999, 1.0, 1.001, 1.7, 3.0, 10.0,
                               33.0, 60.0])
def test_e1_matches_library(direct_oracle, x):
    """E1 by series (x<1, Eq. A.4) and continued fraction (x>=1, Eq. A.2) vs scipy's exp1."""
    assert direct_oracle.e1(x) == pytest.approx(special.exp1(x), rel=5e-15, abs=0)


def test_g_limit_and_continuity(direct_oracle):
    """gamma + log u + E1(u) -> 0 as u -> 0 (Eq. A.5), ~u for small u, continuous at u=1."""
    assert direct_oracle.g0(0.0) == 0.0
    for u in (1e-14, 1e-10, 1e-6):
        assert direct_oracle.g0(u) == pytest.approx(u, rel=1e-5)
    lo = direct_oracle.g0(1.0 - 1e-13)
    hi = direct_oracle.g0(1.0)
    assert abs(hi - lo) < 1e-12
    for u in (0.25, 0.9, 2.0, 40.0):
        assert direct_oracle.g0(u) == pytest.approx(np.euler_gamma + math.log(u) + special.exp1(u),
                                                     rel=1e-13)


KINC_CASES = [(0.154, 0.0), (0.154, 1e-6), (0.154, 3.0), (0.154, 800.0), (0.617, 25.0),
              (2.0, 2.0), (40.0, 0.1), (1e-3, 1e-3), (7.5, 300.0), (0.05, 60.0)]


@pytest.mark.parametrize("a,b", KINC_CASES)
def test_kinc_against_adaptive_quadrature(direct_oracle, a, b):
    """K0(a,b) = int_1^inf t^-1 e^{-at-b/t} dt, by scipy's adaptive quadrature."""
    ref = integrate.quad(lambda t: math.exp(-a * t - b / t) / t, 1.0, np.inf, epsabs=1e-300,
                         epsrel=2e-14, limit=1000)[0]
    assert direct_oracle.kinc(a, b) == pytest.approx(ref, rel=1e-13)
    refd = integrate.quad(lambda t: math.exp(-a * t - b / t) / (t * t), 1.0, np.inf, epsabs=1e-300,
                          epsrel=2e-14, limit=1000)[0]
    assert direct_oracle.kinc_mdb(a, b) == pytest.approx(refd, rel=1e-13)


@pytest.mark.parametrize("a,b", [(0.3, 0.7), (1.2, 0.4), (5.0, 20.0), (0.02, 3.0), (10.0, 10.0)])
def test_kinc_reflection_identity(direct_oracle, a, b):
    """K0(a,b) + K0(b,a) = 2 K_0(2 sqrt(ab)) (Appendix A) with scipy's modified Bessel K_0."""
    lhs = direct_oracle.kinc(a, b) + direct_oracle.kinc(b, a)
    assert lhs == pytest.approx(2.0 * special.k0(2.0 * math.sqrt(a * b)), rel=1e-14)


@pytest.mark.parametrize("a", [0.01, 0.154, 1.0, 9.0])
def test_kinc_at_zero_b_is_e1(direct_oracle, a):
    assert direct_oracle.kinc(a, 0.0) == pytest.approx(special.exp1(a), rel=1e-14)


def test_kinc_derivative_by_finite_difference(direct_oracle):
    for a, b in [(0.154, 2.0), (0.6, 30.0), (3.0, 0.5)]:
        e = 1e-5 * b
        fd = (direct_oracle.kinc(a, b + e) - direct_oracle.kinc(a, b - e)) / (2 * e)
        assert -fd == pytest.approx(direct_oracle.kinc_mdb(a, b), rel=1e-8)


# ---------------------------------------------------------------- Section 4.2 closed forms

@pytest.mark.parametrize("k3", [1.0, 2.0, 3.0])
@pytest.mark.parametrize("hstep", [0.5, 1.0, 2.0])
def test_theorem_4_2_trapezoid_error_identity(k3, hstep):
    """|T_h - F| = (2 pi/k3)/(e^{2 pi k3/h} - 1) (Eq. 4.5) with F = (pi/k3) erfc(sqrt(alpha) k3).

    The residue argument of the proof drops the Gaussian's own aliasing term, of order
    e^{-pi^2/(alpha h^2)} (about 1e-12 at h = 2), so the identity is checked to that level."""
    alpha = 0.1
    j = np.arange(-4000, 4001)
    kk = j * hstep
    T = hstep * np.sum(np.exp(-alpha * (kk * kk + k3 * k3)) / (kk * kk + k3 * k3))
    F1 = math.pi / k3 * math.erfc(math.sqrt(alpha) * k3)
    expect = (2.0 * math.pi / k3) / math.expm1(2.0 * math.pi * k3 / hstep)
    assert abs(T - F1) == pytest.approx(expect, rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("k3", [1.0, 2.5])
def test_two_variable_integral_is_pi_e1(direct_oracle, k3):
    """F2 = int_R2 e^{-alpha(k^2+k3^2)}/(k^2+k3^2) = pi E1(alpha k3^2) (Section 4.2)."""
    alpha = 0.1
    radial = integrate.quad(lambda k: 2 * math.pi * k * math.exp(-alpha * (k * k + k3 * k3))
                            / (k * k + k3 * k3), 0, np.inf, epsrel=1e-13)[0]
    assert radial == pytest.approx(math.pi * direct_oracle.e1(alpha * k3 * k3), rel=1e-12)


# ---------------------------------------------------------------- total potential of the direct sums

def _line_potential(x, q, L3, J=600):
    """Neutral sum of regularised line potentials (Poisson summation of the z images).

    V(rho,dz) = -(2/L3)(log(rho/(2 L3)) + gamma) + (4/L3) sum_j K_0(2 pi j rho/L3) cos(2 pi j dz/L3)
    """
    n = x.shape[0]
    phi = np.zeros(n)
    j = np.arange(1, J + 1)
    for m in range(n):
        for k in range(n):
            if k == m:
                continue
            d = x[m] - x[k]
            rho = math.hypot(d[0], d[1])
            v = (-(2.0 / L3) * (math.log(rho / (2.0 * L3)) + np.euler_gamma)
                 + (4.0 / L3) * np.sum(special.k0(2 * np.pi * j * rho / L3)
                                       * np.cos(2 * np.pi * j * d[2] / L3)))
            phi[m] += q[k] * v
    return phi


def _tiny_system(seed=5, n=6, L3=1.0):
    rng = np.random.default_rng(seed)
    x = rng.random((n, 3)) * np.array([1.0, 1.0, L3])
    q = rng.uniform(-1, 1, n)
    q -= q.mean()
    return x, q


@pytest.mark.parametrize("xi", [4.0, 8.0, 16.0])
def test_total_potential_matches_line_sums(direct_oracle, xi):
    """phi^R+phi^F+phi^self (converged rc, xi rc = 6.5) equals the closed-form line sums,
    at three splitting parameters (so phi is also xi-independent)."""
    x, q = _tiny_system()
    phi, F, U = direct_oracle.ewald1p(x, q, 1.0, xi, 6.5 / xi)
    ref = _line_potential(x, q, 1.0)
    assert np.max(np.abs(phi - ref)) < 1e-12 * np.max(np.abs(ref))


def test_total_potential_matches_brute_force_images(direct_oracle):
    """Direct image sums |alpha| <= A, extrapolated in 1/A (A = 1000..8000)."""
    rng = np.random.default_rng(7)
    L3 = 1.3
    x = rng.random((4, 3)) * np.array([1.0, 1.0, L3])
    q = np.array([1.0, -0.5, 0.75, -1.25])
    n = 4

    def brute(A):
        al = np.arange(-A, A + 1)
        out = np.zeros(n)
        for m in range(n):
            d = x[m] - x
            r = np.sqrt((d[:, 0] ** 2 + d[:, 1] ** 2)[None, :] + (d[:, 2][None, :] + al[:, None] * L3) ** 2)
            r[A, m] = np.inf
            S = (q[None, :] / r).sum(axis=1)
            out[m] = np.sum(S[np.argsort(-np.abs(al))])
        return out

    As = [1000, 2000, 4000, 8000]
    vals = np.array([brute(A) for A in As])
    design = np.array([[1.0, A ** -2.0, A ** -3.0, A ** -4.0] for A in As])
    extrap = np.linalg.solve(design, vals)[0]
    phi, _, _ = direct_oracle.ewald1p(x, q, L3, 6.0, 6.5 / 6.0)
    assert np.max(np.abs(phi - extrap)) < 1e-12


def test_homogeneity_and_z_translation(direct_oracle):
    """L -> lam L, xi -> xi/lam gives phi -> phi/lam, F -> F/lam^2; z shifts of all charges, or of
    single charges by whole periods, change nothing (the sums run over every z image, Eq. 2.2)."""
    x, q = _tiny_system(seed=11, n=8)
    xi = 7.0
    phi, F, _ = direct_oracle.ewald1p(x, q, 1.0, xi, 6.5 / xi)
    lam = 2.5
    phi2, F2, _ = direct_oracle.ewald1p(lam * x, q, lam, xi / lam, 6.5 * lam / xi)
    assert np.max(np.abs(phi2 * lam - phi)) < 1e-12 * np.max(np.abs(phi))
    assert np.max(np.abs(F2 * lam * lam - F)) < 1e-11 * np.max(np.abs(F))
    xs = x.copy()
    xs[:, 2] = np.mod(xs[:, 2] + 0.37, 1.0)
    phi3, F3, _ = direct_oracle.ewald1p(xs, q, 1.0, xi, 6.5 / xi)
    assert np.max(np.abs(phi3 - phi)) < 1e-12 * np.max(np.abs(phi))
    assert np.max(np.abs(F3 - F)) < 1e-11 * np.max(np.abs(F))
    # single charges given at other periodic images (z off by whole periods) change nothing
    xp = x.copy()
    xp[:, 2] += np.array([0, -1, 2, 0, 3, -2, 1, 0])[: len(q)] * 1.0
    phi4, F4, _ = direct_oracle.ewald1p(xp, q, 1.0, xi, 6.5 / xi)
    assert np.max(np.abs(phi4 - phi)) < 1e-12 * np.max(np.abs(phi))
    assert np.max(np.abs(F4 - F)) < 1e-11 * np.max(np.abs(F))


# ---------------------------------------------------------------- forces

def _phi_parts_at(direct_oracle, x, q, m, xi, rc, L3):
    p, _ = direct_oracle.ewald1p_parts(x, q, L3, xi, rc, targets=[m])
    return p[0]


@pytest.mark.parametrize("m", [0, 3])
def test_force_parts_are_minus_q_grad_phi(direct_oracle, m):
    """Each force part (Eqs. 3.22-3.24 read as -q grad phi) equals central differences of
    the matching potential part; pins the 2/L3 factor of the k3=0 force."""
    x, q = _tiny_system(seed=3, n=6, L3=1.2)
    xi, L3 = 5.0, 1.2
    rc = 6.5 / xi
    _, frc = direct_oracle.ewald1p_parts(x, q, L3, xi, rc, targets=[m])
    eps = 1e-5
    for d in range(3):
        xp = x.copy()
        xm = x.copy()
        xp[m, d] += eps
        xm[m, d] -= eps
        dphi = (_phi_parts_at(direct_oracle, xp, q, m, xi, rc, L3)
                - _phi_parts_at(direct_oracle, xm, q, m, xi, rc, L3)) / (2 * eps)
        for part in range(3):
            expect = -q[m] * dphi[part]
            assert frc[0, part, d] == pytest.approx(expect, rel=1e-7, abs=1e-9)


def test_net_force_zero_and_pair_symmetry(direct_oracle):
    x, q = _tiny_system(seed=9, n=10)
    _, F, U = direct_oracle.ewald1p(x, q, 1.0, 6.0, 6.5 / 6.0)
    assert np.max(np.abs(F.sum(axis=0))) < 1e-11 * np.max(np.abs(F))
    x2 = np.array([[0.3, 0.4, 0.1], [0.6, 0.55, 0.7]])
    q2 = np.array([1.0, -1.0])
    _, F2, _ = direct_oracle.ewald1p(x2, q2, 1.0, 6.0, 6.5 / 6.0)
    assert np.max(np.abs(F2[0] + F2[1])) < 1e-12 * np.max(np.abs(F2))


def test_energy_gradient_is_minus_force(direct_oracle):
    """U = 1/2 sum q phi; dU/dx_m = -F_m (reading A1 of the energy)."""
    x, q = _tiny_system(seed=12, n=6)
    xi = 6.0
    _, F, U = direct_oracle.ewald1p(x, q, 1.0, xi, 6.5 / xi)
    eps = 1e-5
    for d in range(3):
        xp = x.copy()
        xm = x.copy()
        xp[2, d] += eps
        xm[2, d] -= eps
        Up = direct_oracle.ewald1p(xp, q, 1.0, xi, 6.5 / xi)[2]
        Um = direct_oracle.ewald1p(xm, q, 1.0, xi, 6.5 / xi)[2]
        assert -(Up - Um) / (2 * eps) == pytest.approx(F[2, d], rel=1e-7)


# ---------------------------------------------------------------- the SE1P algorithm restatement

def test_vico_kernel_is_hankel_transform_of_truncated_log():
    """Eq. 3.9: G_R(kappa) = 2 pi int_0^R J0(kappa r) (-log r / 2 pi) r dr; Eq. 3.10 at 0."""
    R = 2.7
    for kap in (0.0, 0.3, 1.0, 4.5, 13.0):
        ref = integrate.quad(lambda r: -special.j0(kap * r) * r * math.log(r), 0, R,
                             epsrel=1e-13, limit=400)[0]
        val = se.vico_green(np.array([kap]), R)[0]
        assert val == pytest.approx(ref, rel=1e-11, abs=1e-13)


def test_window_integrates_to_one():
    """h sum_g W_1d(x - g h) = 1 up to the truncation/resolution error (Theorem 4.1)."""
    P, xi, h = 24, 8.0, 1.0 / 40
    eta = se.eta_of(P, xi, h)
    for xpos in (0.3, 0.3117, 0.74):
        idx, d = se.support(np.array([xpos]), h, P)
        s = h * se.window_1d(d, xi, eta).sum()
        assert abs(s - 1.0) < 1e-12


def _kspace_direct(direct_oracle, x, q, L3, xi):
    p, f = direct_oracle.ewald1p_parts(x, q, L3, xi, -1.0)
    return p[:, 1] + p[:, 2], f[:, 1] + f[:, 2]


def test_se_algorithm_matches_direct_sums_cubic(direct_oracle):
    """Algorithm 1 at high accuracy (P=24, s_l=4, n_l=6) reproduces Eq. 2.3b + Eq. 2.4."""
    rng = np.random.default_rng(21)
    n = 200
    x = rng.random((n, 3))
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    phi_ref, F_ref = _kspace_direct(direct_oracle, x, q, 1.0, 8.0)
    phi, F = se.se1p_fourier(x, q, (1.0, 1.0, 1.0), 8.0, (40, 40, 40), 24, 64, 192, 256, 6)
    assert rel_rms(phi, phi_ref) < 1e-12
    assert rel_rms(F, F_ref) < 1e-11


def test_se_algorithm_matches_direct_sums_unequal_spacing(direct_oracle):
    """Non-cubic box with a different z spacing: per-axis eta (reading A8) and the I set
    measured in free-direction units (reading A10).  The lowest mode k3 = 2 pi/1.6 is
    harder than 2 pi/L (Section 4.2: error ~ e^{-|k3| s_l Lt}), so s_l = 5 here."""
    rng = np.random.default_rng(22)
    n = 120
    L = (1.0, 1.0, 1.6)
    x = rng.random((n, 3)) * np.array(L)
    q = rng.uniform(-1, 1, n)
    q -= q.mean()
    phi_ref, F_ref = _kspace_direct(direct_oracle, x, q, L[2], 8.0)
    phi, F = se.se1p_fourier(x, q, L, 8.0, (40, 40, 56), 24, 64, 192, 320, 6)
    assert rel_rms(phi, phi_ref) < 1e-11
    assert rel_rms(F, F_ref) < 1e-10


def test_se_algorithm_odd_support(direct_oracle):
    """Odd P (Theorem 4.1's setting) centres the support on round(x/h) (reading A5/A6)."""
    rng = np.random.default_rng(23)
    n = 100
    x = rng.random((n, 3))
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    phi_ref, F_ref = _kspace_direct(direct_oracle, x, q, 1.0, 8.0)
    phi, F = se.se1p_fourier(x, q, (1.0, 1.0, 1.0), 8.0, (40, 40, 40), 25, 66, 198, 264, 6)
    assert rel_rms(phi, phi_ref) < 1e-11
    assert rel_rms(F, F_ref) < 1e-10


def test_se_algorithm_short_periodic_axis(direct_oracle):
    """A periodic axis as short as the support (M3 = P = 20, L3 = 0.5): every window wraps
    around the whole z axis (Eq. 3.7 taken periodically) and still reproduces Eq. 2.3b + Eq. 2.4.
    The discrete operator is symmetric (the same window spreads and gathers, Eqs. 3.7, 3.11), so
    c . phi[q] = q . phi[c] for any two charge vectors."""
    rng = np.random.default_rng(24)
    n = 120
    L = (1.0, 1.0, 0.5)
    x = rng.random((n, 3)) * np.array(L)
    q = rng.uniform(-1, 1, n)
    q -= q.mean()
    phi_ref, F_ref = _kspace_direct(direct_oracle, x, q, L[2], 8.0)
    phi, F = se.se1p_fourier(x, q, L, 8.0, (40, 40, 20), 20, 64, 192, 192, 6)
    assert rel_rms(phi, phi_ref) < 1e-11
    assert rel_rms(F, F_ref) < 1e-10
    c = rng.standard_normal(n)
    c -= c.mean()
    phi_c, _ = se.se1p_fourier(x, c, L, 8.0, (40, 40, 20), 20, 64, 192, 192, 6)
    assert abs(c @ phi - q @ phi_c) < 1e-12 * np.abs(c) @ np.abs(phi)


def test_table_4_1_error_levels(direct_oracle):
    """Table 4.1: parameters for N=120, L=10, Q=1 give absolute rms k-space errors of
    5.4e-7, 9.4e-7, 6.7e-13, 8.3e-13.  Positions are not printed, so only the order of
    magnitude is compared (a factor 10 either way)."""
    with open(os.path.join(GOLDEN, "table_4_1.json")) as f:
        tab = json.load(f)
    rng = np.random.default_rng(41)
    n, L = 120, 10.0
    x = rng.random((n, 3)) * L
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0) / math.sqrt(n)  # Q = sum q^2 = 1
    for xi, M, P, Mt, nl, sl, nI, n0, rms in tab["rows"]:
        phi_ref, _ = _kspace_direct(direct_oracle, x, q, L, xi)
        phi, _ = se.se1p_fourier(x, q, (L, L, L), xi, (M, M, M), P, Mt, n0, nI, nl)
        err = float(np.sqrt(np.mean((phi - phi_ref) ** 2)))
        if rms > 1e-10:
            assert rms / 10 < err < rms * 10, (xi, M, P, err, rms)
        else:
            assert err < rms * 10, (xi, M, P, err, rms)
