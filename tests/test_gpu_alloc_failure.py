"""Plan creation when an allocation fails part-way: SE1P_ERR_ALLOC, no plan, nothing leaked.

The library's test hook SE1P_TEST_FAIL_ALLOC=k makes the k-th workspace allocation of a plan
creation fail as if the device (or the page-locked host pool) were exhausted.  Every k from the
first allocation to the last is tried; each must return SE1P_ERR_ALLOC with a NULL plan and leave
the device's free memory where it was, and a plan created afterwards without the hook must work.
"""
import ctypes
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1611_09538_gb300 import build as se1p_build  # noqa: E402
from paper_1611_09538_gb300 import inputs, se1p  # noqa: E402


@pytest.mark.parametrize("precision,flags", [(se1p.SE1P_MIXED, 0), (se1p.SE1P_FP64, 0),
                                             (se1p.SE1P_MIXED, se1p.SE1P_FLAG_TRIPLY_PERIODIC)])
def test_every_failed_allocation_is_reported_and_freed(precision, flags):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    se1p_build.build()
    lib = se1p.load()
    prm = se1p.make_params((1.0, 1.0, 1.0), 8.0, (32, 32, 32), 16, rc=0.3, precision=precision, flags=flags)
    # one full creation first, so that the library's kernels are loaded (module loading takes device
    # memory of its own, once) before the free memory is recorded
    h = ctypes.c_void_p()
    assert lib.se1p_plan_create(ctypes.byref(prm), 2000, ctypes.byref(h)) == 0
    lib.se1p_plan_destroy(h)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    try:
        for k in range(1, 200):
            os.environ["SE1P_TEST_FAIL_ALLOC"] = str(k)
            h = ctypes.c_void_p()
            code = lib.se1p_plan_create(ctypes.byref(prm), 2000, ctypes.byref(h))
            if code == 0:  # k is beyond the last allocation: creation succeeds
                lib.se1p_plan_destroy(h)
                break
            assert code == 4, (k, se1p.STATUS.get(code))
            assert h.value is None
            failed += 1
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0, k
    finally:
        del os.environ["SE1P_TEST_FAIL_ALLOC"]
    assert failed >= 20  # every buffer of the workspace was tried
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # and without the hook the same parameters give a working plan
    x, q = inputs.uniform_alternating(1000, seed=0)
    plan = se1p.Plan.from_params(prm, 1000)
    r = plan.eval(torch.as_tensor(x, device="cuda"), torch.as_tensor(q, device="cuda"))
    assert np.isfinite(r.phi.cpu().numpy()).all()
    plan.close()
