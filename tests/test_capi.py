"""The C-ABI library loads on a machine without a GPU and exports every declared symbol."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(cp_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1005_3609_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_headers_declare_the_boundary():
    names = declared_functions()
    for need in ("cp_create_strip", "cp_advance_rows", "cp_read_coeffs", "cp_destroy", "cp_crt", "cp_last_error"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1005_3609_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_constants_match_header():
    from paper_1005_3609_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "cp_tm.h")).read()
    assert "#define CP_MAX_L %d" % _lib.CP_MAX_L in src
    assert "#define CP_MAX_PRIMES %d" % _lib.CP_MAX_PRIMES in src
    for code, name in _lib.STATUS.items():
        assert re.search(r"%s = %d\b" % (name, code), src), name


def test_argument_errors_without_gpu(lib):
    # validation happens before any CUDA call
    import ctypes
    from paper_1005_3609_gb300 import _lib
    h = ctypes.c_void_p()
    primes = (ctypes.c_uint32 * 2)(1073741827, 1073741827)
    assert lib.cp_create_strip(0, 0, primes, 1, -1, 2, None, ctypes.byref(h)) == -1
    assert lib.cp_create_strip(0, 21, primes, 1, -1, 2, None, ctypes.byref(h)) == -1
    assert lib.cp_create_strip(2, 4, primes, 1, -1, 2, None, ctypes.byref(h)) == -1
    assert lib.cp_create_strip(0, 4, primes, 2, -1, 2, None, ctypes.byref(h)) == -1   # duplicate
    bad = (ctypes.c_uint32 * 1)(1073741825)                                          # 5 * 214748365
    assert lib.cp_create_strip(0, 4, bad, 1, -1, 2, None, ctypes.byref(h)) == -1
    assert b"prime" in lib.cp_last_error()
    assert lib.cp_advance_rows(None, 1) == -1


def test_newer_entry_points_validate_without_gpu(lib):
    # the Potts strip, the pairing switch and the work queries check their arguments first
    import ctypes
    from paper_1005_3609_gb300 import _lib
    h = ctypes.c_void_p()
    one = (ctypes.c_uint32 * 1)(1073741827)
    src = open(os.path.join(ROOT, "include", "cp_tm.h")).read()
    vmax = int(re.search(r"#define CP_POTTS_MAX_V (\d+)", src).group(1))
    lmax = int(re.search(r"#define CP_POTTS_MAX_L (\d+)", src).group(1))
    assert lib.cp_create_strip_potts(0, 4, vmax + 1, one, 1, -1, 2, None, ctypes.byref(h)) == -1
    assert b"v must be" in lib.cp_last_error()
    assert lib.cp_create_strip_potts(1, lmax + 1, 2, one, 1, -1, 2, None, ctypes.byref(h)) == -1
    assert lib.cp_create_strip_potts(2, 4, 2, one, 1, -1, 2, None, ctypes.byref(h)) == -1  # lattice
    assert lib.cp_create_strip_potts(0, 4, 2, one, 1, -1, 0, None, ctypes.byref(h)) == -1  # max_rows
    assert lib.cp_strip_work(None, (ctypes.c_uint64 * 6)()) == -1
    assert lib.cp_sweep_work(None, (ctypes.c_uint64 * 3)()) == -1
    # the pairing switch returns the previous mode and clamps to 0..3
    old = lib.cp_set_factor_pairing(0)
    assert old in (0, 1, 2, 3)
    assert lib.cp_set_factor_pairing(7) == 0
    assert lib.cp_set_factor_pairing(old) == 3


def test_whitney_bits_on_host(lib):
    import math
    from paper_1005_3609_gb300 import _lib
    for lattice, L, N in (("square", 12, 13), ("triangular", 13, 14), ("square", 1, 1), ("square", 3, 1)):
        e = L * (N - 1) + N * (L - 1) + ((L - 1) * (N - 1) if lattice == "triangular" else 0)
        n = L * N + 3
        assert _lib.whitney_bits(lattice, L, N, n) == [math.comb(e, j).bit_length() for j in range(n)]
