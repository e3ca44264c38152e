"""The FP32 erfc used by the mixed-precision real-space kernel.

erfc(x) = exp(-x^2) erfcx(x) with erfcx fitted by csrc/gen_erfcx_fit.py.  Checks
that the constants compiled into se1p_real.cu are the generator's, and that the
kernel's FP32 evaluation order stays within 4e-7 of scipy's erfcx over [0, 7]
(CUDA's own erfcf is specified to 4 ulp, about 2.4e-7)."""
import importlib.util
import os
import re

import numpy as np
from scipy import special

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1611_09538_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_erfcx_fit", os.path.join(CSRC, "gen_erfcx_fit.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _kernel_constants():
    src = open(os.path.join(CSRC, "se1p_real.cu")).read()
    body = re.search(r"const float c\[11\] = \{([^}]*)\}", src).group(1)
    c = np.array([float(v.strip().rstrip("f")) for v in body.split(",")])
    p = float(re.search(r"kErfcxP = ([0-9.e+-]+)f", src).group(1))
    tc = float(re.search(r"kErfcxTc = ([0-9.e+-]+)f", src).group(1))
    return c, p, tc


def test_kernel_constants_are_the_generators():
    gen = _gen()
    c_gen, _ = gen.fit()
    c_k, p, tc = _kernel_constants()
    assert p == gen.P_SUB
    assert abs(tc - gen.T_C) < 1e-9
    assert np.allclose(c_k, c_gen, rtol=2e-9, atol=1e-12)


def test_fp32_evaluation_error_bound():
    gen = _gen()
    c_k, p, _ = _kernel_constants()
    x = np.linspace(0.0, 7.0, 400001)
    r = gen.eval_fp32(c_k, x, p)
    assert np.abs(r / special.erfcx(x) - 1.0).max() < 4e-7
    # erfc itself, times exp(-x^2) from an FP32 argument: x^2 carries a rounding of
    # x^2 2^-24 in the exponent, so the relative error grows to ~1.5e-6 at x = 4, where
    # erfc(x) < 2e-8 and the pair term is negligible next to the near pairs.
    e = (np.exp(-(x.astype(np.float32) ** 2)).astype(np.float32) * r).astype(np.float64)
    rel = np.abs(e / special.erfc(x) - 1.0)
    assert rel[x <= 1.0].max() < 6e-7
    assert rel[x <= 4.0].max() < 2e-6
