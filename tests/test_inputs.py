"""The seeded input generators (CPU): the bytes both the CUDA path and the oracle consume.

Each generator is deterministic for its seed, keeps positions in the box the plan accepts
(x, y in [0, L), z in [0, L3)), and returns a neutral system (|sum q| <= 1e-12 sum |q|, the plan's
check); the named workloads carry the parameters their documentation states."""
import numpy as np
import pytest

from paper_1611_09538_gb300 import inputs


def check_system(x, q, L, n):
    assert x.shape == (n, 3) and q.shape == (n,)
    assert x.dtype == np.float64 and q.dtype == np.float64
    for a in range(3):
        assert np.all(x[:, a] >= 0.0) and np.all(x[:, a] < L[a])
    assert abs(q.sum()) <= 1e-12 * np.abs(q).sum()


@pytest.mark.parametrize("gen,kw", [
    (inputs.uniform_alternating, dict(n=1001, L=(1.0, 1.0, 1.3))),
    (inputs.uniform_shifted, dict(n=777, L=(2.0, 2.0, 0.5))),
    (inputs.clustered, dict(n=5000, L=(1.0, 1.0, 2.0))),
])
def test_generators_are_seeded_in_box_and_neutral(gen, kw):
    x1, q1 = gen(seed=11, **kw)
    x2, q2 = gen(seed=11, **kw)
    x3, _ = gen(seed=12, **kw)
    assert np.array_equal(x1, x2) and np.array_equal(q1, q2)
    assert not np.array_equal(x1, x3)
    check_system(x1, q1, kw["L"], kw["n"])


@pytest.mark.parametrize("n", [300, 301, 4800])
def test_cloud_wall_stand_in(n):
    L = 10.0
    x, q = inputs.cloud_wall_like(n, L, seed=5)
    check_system(x, q, (L, L, L), n)
    wall = q > 0
    # the wall sits at x = L/2 with thickness 0.01 L; the cloud is centred at x = L/4
    assert abs(np.mean(x[wall, 0]) - L / 2) < 0.01 * L
    assert abs(np.mean(x[q < 0, 0]) - L / 4) < 0.05 * L


def test_batch_systems_ranges():
    systems = inputs.batch_systems(count=16, n_lo=1000, n_hi=50000, seed=4)
    assert len(systems) == 16
    for s in systems:
        n = len(s.q)
        assert 1000 <= n <= 50000 and n % 2 == 0
        assert s.L[0] == s.L[1] == 1.0 and 1.0 <= s.L[2] <= 4.0
        check_system(s.x, s.q, s.L, n)


def test_named_workloads():
    c2 = inputs.config_c2()
    assert len(c2.q) == 100_000 and c2.L == (1.0, 1.0, 1.0)
    assert c2.params == dict(xi=20.0, M=(64, 64, 64), P=24, Mt=96, n0=288, nI=192, nl=4, rc=0.15)
    check_system(c2.x, c2.q, c2.L, 100_000)
    c3 = inputs.config_c3_resolved(n=20_000)
    assert c3.L == (1.0, 1.0, 8.0) and c3.params["M"] == (128, 128, 1024) and c3.params["P"] == 24
    check_system(c3.x, c3.q, c3.L, 20_000)
    c4 = inputs.config_c4(n=20_000)
    assert c4.L == (1.0, 1.0, 2.0) and c4.params["nI"] == 384
    check_system(c4.x, c4.q, c4.L, 20_000)
    for s in (inputs.parity_p0(), inputs.config_c1()):
        assert len(s.q) == 1000
        check_system(s.x, s.q, s.L, 1000)
    # every named grid satisfies the plan's constraints: Mt >= M + P, padded sizes >= Mt
    for s in (inputs.parity_p0(), inputs.config_c1(), c2, c3, c4):
        p = s.params
        assert p["Mt"] >= p["M"][0] + p["P"] and p["n0"] >= p["Mt"] and p["nI"] >= p["Mt"]
        assert p["P"] <= min(p["M"]) and 0 < p["rc"] <= s.L[2]
