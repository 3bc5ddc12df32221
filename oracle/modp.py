"""ctypes wrapper of the plain-C mod-p oracle (``oracle/modp.c``).

Test infrastructure only (see ``oracle/__init__``).  The shared object is
compiled by ``build()`` (gcc, no GPU), here or on any host.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle_modp.so")
_lib = None


def build(force=False):
    src = os.path.join(_HERE, "modp.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", tmp])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.oracle_ptilde_heights.restype = ctypes.c_int
        lib.oracle_ptilde_heights.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
            ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]
        _lib = lib
    return _lib


LATTICE = {"square": 0, "triangular": 1}


def ptilde_heights(lattice, L, heights, D, p):
    """{s: uint32 array of P~(L x s) mod p, coefficients w^0..w^D}."""
    lib = _load()
    hs = sorted(set(int(h) for h in heights))
    arr = (ctypes.c_int * len(hs))(*hs)
    out = np.zeros((len(hs), D + 1), dtype=np.uint32)
    rc = lib.oracle_ptilde_heights(LATTICE[lattice], int(L), arr, len(hs), int(D), int(p),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    if rc != 0:
        raise RuntimeError("oracle_ptilde_heights failed")
    return {h: out[k].copy() for k, h in enumerate(hs)}


def ptilde(lattice, L, N, D, p):
    return ptilde_heights(lattice, L, [N], D, p)[N]
