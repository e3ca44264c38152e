"""Generate the FP32 approximation of erfc used by the real-space kernel.

erfc(x) = exp(-x^2) * erfcx(x), and erfcx is smooth and bounded on [0, X].
With t = 1 / (1 + p x) (the substitution of the classical rational erfc
approximations, e.g. Abramowitz & Stegun 7.1.26 and Hastings) and the centred
variable u = t - tc, tc the midpoint of t's range, erfcx(x) is fitted as
t * (c0 + c1 u + ... + cK u^K) by iteratively reweighted least squares on the
relative error (towards minimax) over x in [0, X].  The kernel
multiplies by exp(-x^2), which it also needs for the force, so one exp serves
both terms and the evaluation has no branches.

Run:  python paper_1611_09538_gb300/csrc/gen_erfcx_fit.py
Prints the constants pasted into se1p_real.cu and the fit's error bounds
(FP64 fit error and FP32-evaluation error), which tests/test_erfc_fit.py
checks again.
"""
from __future__ import annotations

import numpy as np
from scipy import special

P_SUB = 0.5
DEGREE = 10
X_MAX = 7.0
T_C = (1.0 + 1.0 / (1.0 + P_SUB * X_MAX)) / 2.0


def fit(p: float = P_SUB, deg: int = DEGREE, xmax: float = X_MAX):
    x = np.linspace(0.0, xmax, 20001)
    t = 1.0 / (1.0 + p * x)
    R = special.erfcx(x)
    u = t - T_C
    A = np.vstack([t * u ** k for k in range(deg + 1)]).T
    w = 1.0 / R
    c, *_ = np.linalg.lstsq(A * w[:, None], R * w, rcond=None)
    for _ in range(40):
        err = (A @ c - R) / R
        w2 = w * (1.0 + 50.0 * np.abs(err) / np.abs(err).max())
        c, *_ = np.linalg.lstsq(A * w2[:, None], R * w2, rcond=None)
    err = (A @ c - R) / R
    return c, float(np.abs(err).max())


def eval_fp32(c, x, p: float = P_SUB):
    """The kernel's evaluation order in float32: t = 1/(1+p x), u = t - tc, the
    degree-10 polynomial in u by Estrin's scheme, times t."""
    f = np.float32
    c = np.asarray(c, dtype=np.float32)
    x = np.asarray(x, dtype=np.float32)
    t = (f(1.0) / (f(p) * x + f(1.0))).astype(f)
    u = (t - f(T_C)).astype(f)
    u2 = (u * u).astype(f)
    u4 = (u2 * u2).astype(f)
    u8 = (u4 * u4).astype(f)
    p01, p23, p45 = c[1] * u + c[0], c[3] * u + c[2], c[5] * u + c[4]
    p67, p89 = c[7] * u + c[6], c[9] * u + c[8]
    q03, q47, q8a = p23 * u2 + p01, p67 * u2 + p45, c[10] * u2 + p89
    acc = (q8a * u8 + (q47 * u4 + q03)).astype(f)
    return (acc * t).astype(f)


if __name__ == "__main__":
    c, e64 = fit()
    xs = np.linspace(0.0, X_MAX, 200001)
    e32 = np.abs(eval_fp32(c, xs) / special.erfcx(xs) - 1.0).max()
    print(f"// p = {P_SUB}, degree {DEGREE}, x in [0, {X_MAX}]: fit error {e64:.2e}, FP32 evaluation {e32:.2e}")
    print(f"constexpr float kErfcxP = {P_SUB}f, kErfcxTc = {T_C:.9e}f;")
    print("constexpr float kErfcxC[%d] = {" % (DEGREE + 1))
    print(",\n".join(f"    {v:.9e}f" for v in c) + "};")
