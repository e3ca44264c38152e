"""Pins of the triply periodic Ewald oracle (oracle/ewald3p_direct.c), the reference for the SE3P
variant the paper compares SE1P with (Section 1, Example 6.5).

The oracle is checked against numbers mathematics fixes: the Madelung constants of two ionic
crystals (the potential at an ion of an infinite periodic lattice), the independence of the total
sum from the splitting parameter xi, and the force as minus the gradient of the energy.  CPU only.
"""
import json
import os

import numpy as np
import pytest

from oracle import direct

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def total(x, q, L, xi, rc=None):
    rc = 6.5 / xi if rc is None else rc
    pp, ff = direct.ewald3p_parts(x, q, L, xi, rc)
    return pp.sum(axis=1), ff.sum(axis=1)


def madelung():
    with open(os.path.join(GOLDEN, "madelung.json")) as f:
        return json.load(f)


def test_rock_salt_madelung_constant():
    """Eight ions of the NaCl unit cell: every +1 ion sits at potential -M/r0, every -1 ion at
    +M/r0, and every ion at a centre of inversion, so no force acts on it."""
    m = madelung()["NaCl"]
    x = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                  [.5, .5, .5], [.5, 0, 0], [0, .5, 0], [0, 0, .5]], dtype=np.float64)
    q = np.array([1, 1, 1, 1, -1, -1, -1, -1], dtype=np.float64)
    for xi in (3.0, 5.0, 8.0):
        phi, F = total(x, q, (1.0, 1.0, 1.0), xi)
        np.testing.assert_allclose(phi, -q * m["M"] / m["r0"], rtol=1e-14, atol=0)
        assert np.max(np.abs(F)) < 1e-12


def test_caesium_chloride_madelung_constant():
    m = madelung()["CsCl"]
    x = np.array([[0, 0, 0], [.5, .5, .5]], dtype=np.float64)
    q = np.array([1.0, -1.0])
    phi, F = total(x, q, (1.0, 1.0, 1.0), 5.0)
    np.testing.assert_allclose(phi, -q * m["M"] / m["r0"], rtol=1e-13, atol=0)
    assert np.max(np.abs(F)) < 1e-12


def test_rock_salt_in_a_supercell_and_a_shifted_origin():
    """The same crystal described by a 2 x 1 x 1 supercell, shifted by an arbitrary vector:
    the potential at every ion is unchanged (the sum depends only on the infinite lattice)."""
    m = madelung()["NaCl"]
    base = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                     [.5, .5, .5], [.5, 0, 0], [0, .5, 0], [0, 0, .5]], dtype=np.float64)
    qb = np.array([1, 1, 1, 1, -1, -1, -1, -1], dtype=np.float64)
    x = np.concatenate([base, base + [1.0, 0, 0]]) + np.array([0.137, 0.291, 0.053])
    q = np.concatenate([qb, qb])
    phi, _ = total(x, q, (2.0, 1.0, 1.0), 4.0)
    np.testing.assert_allclose(phi, -q * m["M"] / m["r0"], rtol=1e-13, atol=0)


@pytest.fixture(scope="module")
def random_system():
    rng = np.random.default_rng(303)
    L = (1.0, 1.3, 0.8)
    x = rng.random((24, 3)) * np.array(L)
    q = rng.uniform(-1, 1, 24)
    q -= q.mean()
    return x, q, L


def test_total_is_independent_of_xi(random_system):
    """The split into real, Fourier and self parts is exact: the total potential and force of a
    neutral system in a non-cubic box agree at three very different xi."""
    x, q, L = random_system
    res = [total(x, q, L, xi) for xi in (3.0, 5.5, 9.0)]
    for phi, F in res[1:]:
        np.testing.assert_allclose(phi, res[0][0], rtol=0, atol=1e-12 * np.max(np.abs(res[0][0])))
        np.testing.assert_allclose(F, res[0][1], rtol=0, atol=1e-11 * np.max(np.abs(res[0][1])))


def test_force_is_minus_energy_gradient(random_system):
    """F_m = -dU/dx_m with U = 1/2 sum q phi, by central differences (h = 1e-5) on three particles
    and all three axes; the real and Fourier parts are checked separately."""
    x, q, L = random_system
    xi, rc = 5.0, 1.3

    def energies(xx):
        pp, _ = direct.ewald3p_parts(xx, q, L, xi, rc)
        return 0.5 * q @ pp[:, 0], 0.5 * q @ pp[:, 1]

    _, ff = direct.ewald3p_parts(x, q, L, xi, rc)
    h = 1e-5
    for m in (0, 7, 19):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[m, d] += h
            xm[m, d] -= h
            (rp, fp), (rm, fm) = energies(xp), energies(xm)
            assert -(rp - rm) / (2 * h) == pytest.approx(ff[m, 0, d], abs=1e-7)
            assert -(fp - fm) / (2 * h) == pytest.approx(ff[m, 1, d], abs=1e-7)


def test_net_force_vanishes(random_system):
    x, q, L = random_system
    _, F = total(x, q, L, 5.0)
    assert np.max(np.abs(F.sum(axis=0))) < 1e-12 * np.max(np.abs(F))
