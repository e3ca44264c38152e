"""The bounded device wait of the z forward pass (pencils loaded by bulk tensor copies).

Every CTA of that pass waits on an mbarrier for its copies, polling at most a fixed number of
times; a CTA that gives up records SE1P_ERR_TIMEOUT in the plan's status word, waits (bounded) for
its copies to land and returns, so the context stays usable.  The test hook SE1P_TEST_SPIN_LIMIT=0
makes every such wait give up at once: the evaluation must report SE1P_ERR_TIMEOUT through
se1p_plan_sync_status, without a fault or a hang, and a plan created afterwards must work.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1611_09538_gb300 import build as se1p_build  # noqa: E402
from paper_1611_09538_gb300 import inputs, se1p  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    se1p_build.build()


def c2_plan(precision, n):
    s = inputs.config_c2(n)
    p = s.params
    return s, se1p.Plan(s.L, p["xi"], p["M"], p["P"], n, Mt=p["Mt"], n0=p["n0"], nI=p["nI"], nl=p["nl"],
                        rc=p["rc"], precision=precision)


@pytest.mark.parametrize("precision", [se1p.SE1P_MIXED, se1p.SE1P_FP64])
def test_c2_z_pass_uses_tensor_copies(precision):
    _, plan = c2_plan(precision, 2000)
    assert plan.info["features"] & 1
    plan.close()


@pytest.mark.parametrize("precision", [se1p.SE1P_MIXED, se1p.SE1P_FP64])
def test_wait_that_gives_up_reports_timeout(precision):
    os.environ["SE1P_TEST_SPIN_LIMIT"] = "0"
    try:
        s, plan = c2_plan(precision, 2000)
    finally:
        del os.environ["SE1P_TEST_SPIN_LIMIT"]
    x = torch.as_tensor(s.x, device="cuda")
    q = torch.as_tensor(s.q, device="cuda")
    plan.eval(x, q, check=False)
    assert se1p.se1p_plan_sync_status(plan.handle) == 6  # SE1P_ERR_TIMEOUT
    plan.close()
    # the context is intact: a fresh plan evaluates and reports success
    _, plan = c2_plan(precision, 2000)
    r = plan.eval(x, q)
    assert np.isfinite(r.phi.cpu().numpy()).all()
    plan.close()
