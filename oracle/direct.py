"""ctypes front end of the FP64 direct Ewald oracles: Ewald1P (ewald1p_direct.c) and, for the
triply periodic comparison method, Ewald3P (ewald3p_direct.c).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The shared object is built
from ewald1p_direct.c by ``build()`` (plain gcc, OpenMP) into oracle/_build.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ewald1p_direct.c")
_SRC3 = os.path.join(_HERE, "ewald3p_direct.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libewald1p_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math) if it is stale."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC3))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, _SRC3, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        lib.orc_e1.restype = d
        lib.orc_e1.argtypes = [d]
        lib.orc_g.restype = d
        lib.orc_g.argtypes = [d]
        lib.orc_kinc.restype = d
        lib.orc_kinc.argtypes = [d, d]
        lib.orc_kinc_mdb.restype = d
        lib.orc_kinc_mdb.argtypes = [d, d]
        lib.orc_ewald1p.restype = i
        lib.orc_ewald1p.argtypes = [i, p, p, i, p, d, d, d, d, p, p]
        lib.orc_ewald3p.restype = i
        lib.orc_ewald3p.argtypes = [i, p, p, i, p, p, d, d, d, p, p]
        lib.orc_num_threads.restype = i
        lib.orc_num_threads.argtypes = []
        _lib = lib
    return _lib


def e1(x: float) -> float:
    return _load().orc_e1(float(x))


def g0(u: float) -> float:
    """gamma + log u + E1(u)."""
    return _load().orc_g(float(u))


def kinc(a: float, b: float) -> float:
    """Incomplete Bessel K0(a,b) = int_1^inf t^-1 exp(-a t - b/t) dt."""
    return _load().orc_kinc(float(a), float(b))


def kinc_mdb(a: float, b: float) -> float:
    """-d K0(a,b) / db = int_1^inf t^-2 exp(-a t - b/t) dt."""
    return _load().orc_kinc_mdb(float(a), float(b))


def num_threads() -> int:
    return _load().orc_num_threads()


def ewald1p_parts(x, q, L3, xi, rc, targets=None, kcut=1e-20):
    """Per-target parts of the Ewald1P potential and force (Section 2.1, Section 3.5).

    Returns (phi_parts [nt,4]: R, F_k3!=0, F_k3=0, self;
             force_parts [nt,3,3]: R, F_k3!=0, F_k3=0).
    """
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    n = x.shape[0]
    if targets is None:
        nt = n
        tptr = None
        tg = None
    else:
        tg = np.ascontiguousarray(targets, dtype=np.int32)
        nt = tg.size
        tptr = tg.ctypes.data
    phi = np.zeros((nt, 4))
    frc = np.zeros((nt, 3, 3))
    rc_arg = float(rc) if rc is not None else -1.0
    rcode = lib.orc_ewald1p(n, x.ctypes.data, q.ctypes.data, nt, tptr, float(L3), float(xi),
                            rc_arg, float(kcut), phi.ctypes.data, frc.ctypes.data)
    if rcode != 0:
        raise ValueError("oracle rejected its arguments")
    return phi, frc


def ewald1p(x, q, L3, xi, rc, targets=None, kcut=1e-20):
    """Total phi [nt], F [nt,3] and U = 1/2 sum q phi (all targets only)."""
    phi_p, frc_p = ewald1p_parts(x, q, L3, xi, rc, targets, kcut)
    phi = phi_p.sum(axis=1)
    F = frc_p.sum(axis=1)
    U = None
    if targets is None:
        U = 0.5 * float(np.dot(np.asarray(q, dtype=np.float64), phi))
    return phi, F, U


def ewald3p_parts(x, q, L, xi, rc, targets=None, kcut=1e-20):
    """Per-target parts of the triply periodic Ewald potential and force (tin-foil boundary).

    Returns (phi_parts [nt,3]: R, F, self; force_parts [nt,2,3]: R, F).  rc <= 0 skips the
    real space."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    Lv = np.ascontiguousarray(L, dtype=np.float64)
    n = x.shape[0]
    if targets is None:
        nt, tptr, tg = n, None, None
    else:
        tg = np.ascontiguousarray(targets, dtype=np.int32)
        nt, tptr = tg.size, tg.ctypes.data
    phi = np.zeros((nt, 3))
    frc = np.zeros((nt, 2, 3))
    rcode = lib.orc_ewald3p(n, x.ctypes.data, q.ctypes.data, nt, tptr, Lv.ctypes.data, float(xi),
                            float(rc) if rc is not None else -1.0, float(kcut), phi.ctypes.data, frc.ctypes.data)
    if rcode != 0:
        raise ValueError("oracle rejected its arguments")
    return phi, frc


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
