"""cp_crt_static: Chinese remaindering without any device allocation.

Callers whose device memory belongs entirely to another allocator, or whose
service forbids new device allocations once it runs, cannot use cp_crt (it
allocates two device buffers per call).  cp_crt_static stages the residues and
limbs in one fixed device array instead.  These tests call it through the C
ABI and compare it with cp_crt on the same inputs, bit for bit (the results are
integers), on two calls in a row: the second call is smaller, so anything the
first call left in the shared array must not leak into it.  The file is named
to be collected last and passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

import gpu_util

pytestmark = pytest.mark.gpu

cp = pytest.importorskip("paper_1005_3609_gb300")
from paper_1005_3609_gb300 import _lib  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _lib.load()


def call(lib, fn, residues, primes, limbs):
    res = np.ascontiguousarray(np.asarray(residues, dtype=np.uint32))
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32))
    out = np.zeros((res.shape[1], limbs), dtype=np.uint32)
    rc = getattr(lib, fn)(res.ctypes.data_as(_lib.u32p), pr.ctypes.data_as(_lib.u32p), len(pr), res.shape[1],
                          out.ctypes.data_as(_lib.u32p), limbs)
    return rc, out


def test_static_crt_matches_allocating_crt_twice(lib):
    rng = np.random.default_rng(11)
    primes16 = gpu_util.seed_primes(16)
    primes5 = gpu_util.seed_primes(5, seed=2)
    # call 1: 16 primes x 20000 coefficients (about 1.3 MB of residues and 1.4 MB of limbs)
    r1 = np.stack([rng.integers(0, p, size=20000, dtype=np.int64) for p in primes16]).astype(np.uint32)
    # call 2: fewer primes and coefficients, and fewer limbs per coefficient
    r2 = np.stack([rng.integers(0, p, size=777, dtype=np.int64) for p in primes5]).astype(np.uint32)
    for res, primes, limbs in ((r1, primes16, 17), (r2, primes5, 6)):
        rc_a, want = call(lib, "cp_crt", res, primes, limbs)
        rc_b, got = call(lib, "cp_crt_static", res, primes, limbs)
        assert rc_a == 0 and rc_b == 0, lib.cp_last_error()
        assert np.array_equal(got, want)
    # and the integers are the right ones: reduce them back modulo each prime
    ints = _lib.limbs_to_ints(got)
    for k, p in enumerate(primes5):
        assert [x % p for x in ints] == [int(v) for v in r2[k]]


def test_static_crt_rejects_oversize(lib):
    primes = gpu_util.seed_primes(16)
    n = (8 << 20) // (4 * 16) + 1  # residues alone exceed the array
    res = np.zeros((16, n), dtype=np.uint32)
    rc, _ = call(lib, "cp_crt_static", res, primes, 17)
    assert rc == -1  # CP_EINVAL
    assert b"CP_CRT_STATIC_BYTES" in lib.cp_last_error()


FRESH = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
import gpu_util
from paper_1005_3609_gb300 import _lib
lib = _lib.load()
primes = gpu_util.seed_primes(6, seed=4)
rng = np.random.default_rng(3)
res = np.stack([rng.integers(0, p, size=4096, dtype=np.int64) for p in primes]).astype(np.uint32)
out = []
for fn in ("cp_crt_static", "cp_crt"):  # the allocation-free call comes first in this process
    o = np.zeros((res.shape[1], 7), dtype=np.uint32)
    rc = getattr(lib, fn)(res.ctypes.data_as(_lib.u32p), np.asarray(primes, dtype=np.uint32).ctypes.data_as(_lib.u32p),
                          len(primes), res.shape[1], o.ctypes.data_as(_lib.u32p), 7)
    assert rc == 0, (fn, lib.cp_last_error())
    out.append(o)
assert np.array_equal(out[0], out[1])
print("fresh ok")
"""


def test_static_crt_first_call_in_a_fresh_process(lib):
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", FRESH, root], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "fresh ok" in r.stdout, r.stdout + r.stderr
