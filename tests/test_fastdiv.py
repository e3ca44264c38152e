"""The multiply-high division constants the Fourier kernels use for their index arithmetic.

make_fastdiv (host side of csrc/se1p_internal.cuh) builds, for a divisor d, the constants (m, l) of
the round-up method of Granlund and Montgomery; the kernels compute floor(x / d) as
(umulhi(m, x) + x) >> l for 0 <= x < 2^31.  A host-only program, compiled with nvcc against the
same header, evaluates that expression (umulhi as the high half of the 64-bit product) and compares
it with exact integer division over every divisor up to 4096 and a spread of larger ones, each with
small, boundary and large numerators.  No GPU is used.
"""
import os
import subprocess

import pytest

from paper_1611_09538_gb300 import build as lib_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1611_09538_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include "se1p_internal.cuh"

static unsigned host_fdiv(unsigned x, const se1p::FastDiv &f)
{
    const unsigned t = (unsigned)(((unsigned long long)x * f.m) >> 32);  // umulhi
    return (t + x) >> f.l;
}

int main()
{
    unsigned long long checked = 0, bad = 0;
    unsigned ds[6000];
    int nd = 0;
    for (unsigned d = 1; d <= 4096; ++d) ds[nd++] = d;
    for (unsigned d = 4097; nd < 6000; d = d + d / 7 + 13) ds[nd++] = d < (1u << 31) ? d : (1u << 31) - 1;
    for (int i = 0; i < nd; ++i) {
        const unsigned d = ds[i];
        const se1p::FastDiv f = se1p::make_fastdiv(d);
        if (f.d != d) ++bad;
        unsigned xs[64];
        int nx = 0;
        for (unsigned k = 0; k < 8; ++k) xs[nx++] = k;
        for (unsigned q = 1; q < 6; ++q) {  // around multiples of d
            const unsigned long long m = (unsigned long long)q * d;
            if (m + 1 < (1ull << 31)) { xs[nx++] = (unsigned)(m - 1); xs[nx++] = (unsigned)m; xs[nx++] = (unsigned)(m + 1); }
        }
        unsigned long long s = 0x9e3779b97f4a7c15ull ^ d;
        while (nx < 60) {  // pseudo-random numerators below 2^31 (xorshift)
            s ^= s << 13; s ^= s >> 7; s ^= s << 17;
            xs[nx++] = (unsigned)(s & 0x7fffffffu);
        }
        xs[nx++] = (1u << 31) - 1;
        for (int j = 0; j < nx; ++j) {
            ++checked;
            if (host_fdiv(xs[j], f) != xs[j] / d) ++bad;
        }
    }
    printf("%llu %llu\n", checked, bad);
    return bad != 0;
}
"""


def test_fastdiv_constants_divide_exactly(tmp_path):
    try:
        nvcc = lib_build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    src = tmp_path / "fastdiv_check.cu"
    exe = tmp_path / "fastdiv_check"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    checked, bad = (int(v) for v in out.stdout.split())
    assert checked > 300_000
    assert bad == 0 and out.returncode == 0
