"""CPU-only checks of the C-ABI library: it builds, loads and exports every
symbol include/se1p.h declares; host-side argument validation needs no GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1611_09538_gb300 import build as se1p_build
from paper_1611_09538_gb300 import se1p

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = se1p_build.build()
    return se1p.load(path)


def declared_symbols():
    with open(os.path.join(ROOT, "include", "se1p.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:se1p_status|const char \*|se1p_plan \*)\s*(se1p_\w+)\s*\(", text, re.M)))


def test_header_and_binding_agree():
    assert sorted(se1p.EXPORTS) == declared_symbols()


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", se1p.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (se1p_\w+)", out))
    for name in declared_symbols():
        assert name in exported, name
        assert hasattr(lib, name)


def test_params_struct_layout():
    assert ctypes.sizeof(se1p.se1p_params) == 104
    assert ctypes.sizeof(se1p.se1p_plan_info) == 96


def test_status_strings(lib):
    for code, name in se1p.STATUS.items():
        assert se1p.se1p_status_string(code) == name


@pytest.mark.parametrize("bad", [
    dict(L=(1, 1, 1), xi=-1.0, M=(32, 32, 32), P=16),       # xi <= 0
    dict(L=(1, 2, 1), xi=8.0, M=(32, 32, 32), P=16),        # unequal free dimensions
    dict(L=(1, 1, 1), xi=8.0, M=(32, 32, 32), P=40),        # P > 32
    dict(L=(1, 1, 1), xi=8.0, M=(32, 32, 22), P=16),        # M3 not 7-smooth
    dict(L=(1, 1, 1), xi=8.0, M=(32, 32, 32), P=16, Mt=40), # Mt < M + P
    dict(L=(1, 1, 1), xi=8.0, M=(32, 32, 32), P=16, n0=143),  # n0 not 7-smooth
    dict(L=(1, 1, 1), xi=8.0, M=(32, 32, 32), P=16, rc=2.0),  # rc > L3
    dict(L=(1, 1, 1), xi=8.0, M=(32, 32, 32), P=16, flags=2),  # unknown flag
    dict(L=(1, 1, 1), xi=8.0, M=(32, 32, 32), P=15, flags=1),  # triply periodic: odd P
    dict(L=(1, 1, 1), xi=8.0, M=(22, 22, 32), P=16, flags=1),  # triply periodic: M not 7-smooth
    dict(L=(0.5, 0.5, 2), xi=8.0, M=(32, 32, 64), P=16, rc=0.8, flags=1),  # triply periodic: rc > L1
])
def test_invalid_parameters_rejected_on_host(lib, bad):
    kw = dict(bad)
    prm = se1p.make_params(kw.pop("L"), kw.pop("xi"), kw.pop("M"), kw.pop("P"), **kw)
    h = ctypes.c_void_p()
    code = lib.se1p_plan_create(ctypes.byref(prm), 100, ctypes.byref(h))
    assert code == 1 and h.value is None


def test_null_arguments_rejected(lib):
    assert lib.se1p_plan_create(None, 10, None) == 1
    assert lib.se1p_eval(None, 0, None, None, None, None, None, None) == 1
    assert lib.se1p_plan_get_info(None, None) == 1
    assert lib.se1p_plan_destroy(None) == 0
