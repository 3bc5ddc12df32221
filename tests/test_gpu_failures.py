"""Failure paths, exercised without faulting or hanging the GPU.

* A bounded device wait that runs out: a diagnostic kernel waits on an mbarrier
  that nothing arrives on, for ~1 ms; the host must see CP_ETIMEOUT and the
  context must still work afterwards.
* Host-side faults of the server: a request over the memory budget is refused,
  a queued request is cancelled, the others still complete correctly.
"""
import pytest

import gpu_util
from oracle import tm_exact

pytestmark = pytest.mark.gpu

cp = pytest.importorskip("paper_1005_3609_gb300")
from paper_1005_3609_gb300 import _lib  # noqa: E402


@pytest.fixture(scope="module")
def stream():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cp.load()
    return torch.cuda.Stream()


def test_bounded_wait_reports_timeout_and_context_survives(stream):
    lib = _lib.load()
    assert lib.cp_debug_wait_timeout(2_000_000) == -4  # CP_ETIMEOUT after ~1 ms of SM clock
    assert b"bounded wait" in lib.cp_last_error()
    # the error word was cleared and the GPU is still usable
    primes = gpu_util.seed_primes(4)
    with cp.Strip("square", 5, primes, max_degree=-1, max_rows=6, stream=stream) as s:
        s.advance(5)
        assert s.read().tolist() == gpu_util.residues_of(tm_exact.ptilde("square", 5, 6), primes)


def test_server_refusal_and_cancellation(stream):
    primes = gpu_util.seed_primes(4)
    with cp.Server(6 << 20, max_active=1, stream=stream) as sv:
        with pytest.raises(cp.CPError):
            sv.submit("square", 12, 13, primes)  # footprint over the whole budget
        a = sv.submit("triangular", 7, 7, primes)
        b = sv.submit("square", 6, 7, primes)
        c = sv.submit("square", 5, 5, primes)
        sv.cancel(b)
        while sv.result(a)[0] != sv.DONE or sv.result(c)[0] != sv.DONE:
            sv.step()
        assert sv.result(b)[0] == sv.FAILED
        with pytest.raises(cp.CPError):
            sv.cancel(a)  # already finished
        assert sv.result(a)[1].tolist() == gpu_util.residues_of(tm_exact.ptilde("triangular", 7, 7), primes)
        assert sv.result(c)[1].tolist() == gpu_util.residues_of(tm_exact.ptilde("square", 5, 5), primes)
