"""Parameter selection (Section 4.3) through the C ABI's host-only se1p_autotune.

Checked against the oracles: on a Table 4.1-like system (N=120, L=10, Q=1) the
chosen parameters must reach the requested tolerance in the k-space potential
(numpy restatement of Algorithm 1 vs the direct sums) and in the real-space
truncation (direct sums at rc vs converged rc)."""
import numpy as np
import pytest

from oracle import direct
from oracle import se1p_algorithm as se
from paper_1611_09538_gb300 import build as se1p_build
from paper_1611_09538_gb300 import se1p


@pytest.fixture(scope="module", autouse=True)
def _lib():
    se1p_build.build()
    se1p.load()


def _system():
    rng = np.random.default_rng(41)
    n, L = 120, 10.0
    x = rng.random((n, 3)) * L
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0) / np.sqrt(n)
    return x, q, L


@pytest.mark.parametrize("xi,tol", [(1.5, 1e-6), (3.0, 1e-6), (1.5, 1e-9), (3.0, 1e-9)])
def test_autotuned_parameters_reach_tolerance(direct_oracle, xi, tol):
    x, q, L = _system()
    p = se1p.se1p_autotune((L, L, L), xi, float(np.sum(q * q)), len(q), tol)
    assert p.M[0] % 2 == 0 and p.P % 2 == 0 and p.P <= 32 and p.Mt >= p.M[0] + p.P
    assert p.n0 >= 2.4 * p.Mt and p.nI >= p.Mt and p.nl >= 1
    pp, _ = direct.ewald1p_parts(x, q, L, xi, -1.0)
    phi, _ = se.se1p_fourier(x, q, (L, L, L), xi, tuple(p.M), p.P, p.Mt, p.n0, p.nI, p.nl)
    assert np.sqrt(np.mean((phi - (pp[:, 1] + pp[:, 2])) ** 2)) < tol
    pr, _ = direct.ewald1p_parts(x, q, L, xi, p.rc)
    pc, _ = direct.ewald1p_parts(x, q, L, xi, 6.5 / xi)
    assert np.sqrt(np.mean((pr[:, 0] - pc[:, 0]) ** 2)) < 2.5 * tol


def test_table_4_1_grid_sizes_at_moderate_accuracy():
    """Table 4.1 rows 1-2 (tol 1e-6): M = 32 and 64, P = 12 within one step of 2."""
    for xi, M, P in ((1.5, 32, 12), (3.0, 64, 12)):
        p = se1p.se1p_autotune((10.0, 10.0, 10.0), xi, 1.0, 120, 1e-6)
        assert abs(p.M[0] - M) <= 0.15 * M
        assert abs(p.P - P) <= 2


def test_elongated_box_upsamples_low_modes():
    """The lowest z mode of a long box (k3 = 2 pi / L3) is integrated with an error that decays
    like exp(-|k3| (s_l Lt - L)) (the nearest images implied by the rule lie s_l Lt - L away,
    Section 4.2), so the upsampled length beyond the box, s_l Lt - L, grows in proportion to L3."""
    p1 = se1p.se1p_autotune((1.0, 1.0, 1.0), 20.0, 1e4, 10000, 1e-6)
    p4 = se1p.se1p_autotune((1.0, 1.0, 4.0), 20.0, 1e4, 10000, 1e-6)
    beyond = lambda p: p.nI / p.M[0] - 1.0  # s_l Lt - L with Lt = Mt h, h = 1 / M
    assert 3.5 < beyond(p4) / beyond(p1) < 4.5
    assert p4.M[2] > 3.5 * p1.M[2] and p4.M[0] == p1.M[0]


@pytest.mark.parametrize("bad", [
    dict(L=(1, 2, 1)), dict(xi=0.0), dict(tol=0.0), dict(tol=1.0), dict(Q=0.0), dict(n=0)])
def test_autotune_rejects_bad_requests(bad):
    kw = dict(L=(1.0, 1.0, 1.0), xi=8.0, Q=10.0, n=100, tol=1e-6)
    kw.update(bad)
    with pytest.raises(se1p.SE1PError) as ei:
        se1p.se1p_autotune(kw["L"], kw["xi"], kw["Q"], kw["n"], kw["tol"])
    assert ei.value.code == 1


def _golden_6_1():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "table_6_1.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("tol", [1e-5, 1e-9])
def test_table_6_1_parameters(tol):
    """Section 6, Table 6.1 (xi = 4, N/L^3 = 125): the recipe's M, rc and s_l as printed.

    k_inf is taken at tol/100 (the estimates of Eq. 2.10 undershoot the measured k-space error),
    so M may exceed the printed grid by the sqrt-log growth of k_inf, at most 15%; rc follows
    Eq. 2.9 at tol itself (printed 0.781 and 1.08); s_l meets exp(-2 pi s_l) <= tol (Eq. 4.8)
    and, because tol is absolute and the quadrature error grows with sqrt(Q/V), lies between the
    printed value and one above it; n_l follows M ~ 10 n_l (Eq. 4.9)."""
    g = _golden_6_1()["table_6_1"]
    key = "1e-5" if tol == 1e-5 else "1e-9"
    for N, L, M5, nl5, M9, nl9 in g["rows"]:
        M_paper = M5 if tol == 1e-5 else M9
        p = se1p.se1p_autotune((L, L, L), g["xi"], float(N) / 3.0, N, tol)
        assert M_paper <= p.M[0] <= 1.15 * M_paper, (N, p.M[0], M_paper)
        assert abs(p.rc / g["rc"][key] - 1.0) < 0.08, (N, p.rc)
        assert np.exp(-2.0 * np.pi * p.sl) <= tol * 1.0001
        assert g["sl"][key] - 0.1 <= p.nI / p.Mt <= g["sl"][key] + 1.0, (N, p.nI / p.Mt)
        assert p.nl == int(np.ceil(p.M[0] / 10.0))
