"""ctypes binding of libcp_gb300.so (argument marshalling only).

Every computation happens in the CUDA library; this module converts Python
arguments to the C ABI of include/cp_tm.h and raises on a negative status.
There is no fallback: if the shared library is missing this raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcp_gb300.so")

CP_SQUARE, CP_TRIANGULAR = 0, 1
LATTICES = {"square": CP_SQUARE, "triangular": CP_TRIANGULAR}
STATUS = {0: "CP_OK", -1: "CP_EINVAL", -2: "CP_ENOMEM", -3: "CP_ECUDA", -4: "CP_ETIMEOUT", -5: "CP_ESTATE",
          -6: "CP_EPRIMES"}
CP_EPRIMES = -6
CP_MAX_L = 20
CP_MAX_PRIMES = 32

u32p = ctypes.POINTER(ctypes.c_uint32)
u64p = ctypes.POINTER(ctypes.c_uint64)
vp = ctypes.c_void_p


class CPError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__("%s -> %s: %s" % (fn, STATUS.get(code, code), msg))
        self.code = code


# name -> (restype, argtypes)
SIGNATURES = {
    "cp_create_strip": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, u32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       vp, ctypes.POINTER(vp)]),
    "cp_create_strip_potts": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]),
    "cp_advance_rows": (ctypes.c_int, [vp, ctypes.c_int]),
    "cp_read_coeffs": (ctypes.c_int, [vp, u32p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int)]),
    "cp_read_coeffs_device": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
    "cp_strip_info": (ctypes.c_int, [vp, u64p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "cp_destroy": (None, [vp]),
    "cp_strip_reset": (ctypes.c_int, [vp]),
    "cp_strip_set_tile": (ctypes.c_int, [vp, ctypes.c_int]),
    "cp_strip_work": (ctypes.c_int, [vp, u64p]),
    "cp_set_factor_pairing": (ctypes.c_int, [ctypes.c_int]),
    "cp_sweep_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, u32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       vp, ctypes.POINTER(vp)]),
    "cp_sweep_run": (ctypes.c_int, [vp]),
    "cp_sweep_sync": (ctypes.c_int, [vp]),
    "cp_sweep_work": (ctypes.c_int, [vp, u64p]),
    "cp_sweep_info": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), u64p, u64p,
                                     ctypes.POINTER(ctypes.c_int)]),
    "cp_sweep_rects": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "cp_sweep_read_ptilde": (ctypes.c_int, [vp, u32p, ctypes.c_size_t]),
    "cp_sweep_read_series": (ctypes.c_int, [vp, u32p, ctypes.c_size_t]),
    "cp_sweep_read_series_device": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
    "cp_sweep_destroy": (None, [vp]),
    "cp_sweep_set_primes": (ctypes.c_int, [vp, u32p, ctypes.c_int]),
    "cp_sweep_profile": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_float)]),
    "cp_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, vp, ctypes.POINTER(vp)]),
    "cp_server_submit": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p, ctypes.c_int, u64p]),
    "cp_server_step": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]),
    "cp_server_result": (ctypes.c_int, [vp, ctypes.c_uint64, u32p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_double)]),
    "cp_server_release": (ctypes.c_int, [vp, ctypes.c_uint64]),
    "cp_server_poll": (ctypes.c_int, [vp, u64p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "cp_server_cancel": (ctypes.c_int, [vp, ctypes.c_uint64]),
    "cp_debug_wait_timeout": (ctypes.c_int, [ctypes.c_longlong]),
    "cp_debug_table": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p,
                                      ctypes.c_uint64, u32p, ctypes.c_uint64, u64p]),
    "cp_debug_reduce": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64), u32p, ctypes.c_int, u32p]),
    "cp_debug_reduce_halves": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), u32p,
                                              ctypes.c_int, ctypes.c_int, u32p]),
    "cp_server_stats": (ctypes.c_int, [vp, u64p, u64p, u64p, ctypes.POINTER(ctypes.c_size_t)]),
    "cp_server_destroy": (None, [vp]),
    "cp_crt": (ctypes.c_int, [u32p, u32p, ctypes.c_int, ctypes.c_int, u32p, ctypes.c_int]),
    "cp_crt_device": (ctypes.c_int, [vp, u32p, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp]),
    "cp_crt_static": (ctypes.c_int, [u32p, u32p, ctypes.c_int, ctypes.c_int, u32p, ctypes.c_int]),
    "cp_crt_checked": (ctypes.c_int, [u32p, u32p, ctypes.c_int, ctypes.c_int, u32p, u32p, ctypes.c_int, u32p]),
    "cp_whitney_bits": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p]),
    "cp_read_integers": (ctypes.c_int, [vp, u32p, ctypes.c_size_t, ctypes.c_int, u32p, ctypes.POINTER(ctypes.c_int)]),
    "cp_sweep_series_integers": (ctypes.c_int, [vp, u32p, ctypes.c_size_t, ctypes.c_int, u32p]),
    "cp_select_primes": (ctypes.c_int, [u64p, ctypes.c_int, ctypes.c_int, u32p]),
    "cp_clear_table_cache": (None, []),
    "cp_last_error": (ctypes.c_char_p, []),
    "cp_debug_check_space": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p, u64p]),
    "cp_debug_enumerate_space": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_uint8), ctypes.c_uint64, u64p]),
}

_lib = None


def load(path=LIB_PATH):
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libcp_gb300.so is not built (%s); run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def check(fn, rc):
    if rc != 0:
        raise CPError(fn, rc, load().cp_last_error().decode(errors="replace"))


def _u32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    return a, a.ctypes.data_as(u32p)


def lattice_id(lattice):
    return LATTICES[lattice] if isinstance(lattice, str) else int(lattice)


def select_primes(draws, n_primes):
    d = np.ascontiguousarray(np.asarray(draws, dtype=np.uint64))
    out = np.zeros(n_primes, dtype=np.uint32)
    check("cp_select_primes", load().cp_select_primes(d.ctypes.data_as(u64p), len(d), n_primes,
                                                      out.ctypes.data_as(u32p)))
    return [int(p) for p in out]


def limbs_to_ints(limbs):
    """Rows of little-endian 32-bit two's-complement limbs -> Python ints."""
    out = []
    nl = limbs.shape[1]
    for row in limbs:
        v = 0
        for l in range(nl - 1, -1, -1):
            v = (v << 32) | int(row[l])
        if v >> (32 * nl - 1):
            v -= 1 << (32 * nl)
        out.append(v)
    return out


def crt(residues, primes, limbs_per_coeff=None):
    """residues [P][n] -> list of n signed integers (cp_crt)."""
    res, rp = _u32(residues)
    pr, pp = _u32(primes)
    P, n = res.shape
    if limbs_per_coeff is None:
        limbs_per_coeff = (31 * P + 2 + 31) // 32 + 1
    out = np.zeros((n, limbs_per_coeff), dtype=np.uint32)
    check("cp_crt", load().cp_crt(rp, pp, P, n, out.ctypes.data_as(u32p), limbs_per_coeff))
    return limbs_to_ints(out)


def limbs_for(n_primes):
    """Limbs per coefficient that hold any value the n_primes primes (< 2^31) determine."""
    return (31 * n_primes + 2 + 31) // 32 + 1


def crt_checked(residues, primes, bound_bits=None, limbs_per_coeff=None):
    """cp_crt_checked: (integers, flags, status) -- status 0 or CP_EPRIMES (too few primes)."""
    res, rp = _u32(residues)
    pr, pp = _u32(primes)
    P, n = res.shape
    limbs_per_coeff = limbs_per_coeff or limbs_for(P)
    out = np.zeros((n, limbs_per_coeff), dtype=np.uint32)
    flags = np.zeros(n, dtype=np.uint32)
    bp = None
    if bound_bits is not None:
        bb, bp = _u32(bound_bits)
    rc = load().cp_crt_checked(rp, pp, P, n, bp, out.ctypes.data_as(u32p), limbs_per_coeff,
                               flags.ctypes.data_as(u32p))
    if rc not in (0, CP_EPRIMES):
        check("cp_crt_checked", rc)
    return limbs_to_ints(out), [int(f) for f in flags], rc


def whitney_bits(lattice, L, N, n_coeffs):
    """Bit lengths of C(|E|, j), j < n_coeffs, for the L x N rectangle (cp_whitney_bits)."""
    out = np.zeros(n_coeffs, dtype=np.uint32)
    check("cp_whitney_bits", load().cp_whitney_bits(lattice_id(lattice), L, N, n_coeffs, out.ctypes.data_as(u32p)))
    return [int(x) for x in out]


def crt_static(residues, primes, limbs_per_coeff=None):
    """As crt(), through cp_crt_static (no device allocation; fixed-size staging array)."""
    res, rp = _u32(residues)
    pr, pp = _u32(primes)
    P, n = res.shape
    if limbs_per_coeff is None:
        limbs_per_coeff = (31 * P + 2 + 31) // 32 + 1
    out = np.zeros((n, limbs_per_coeff), dtype=np.uint32)
    check("cp_crt_static", load().cp_crt_static(rp, pp, P, n, out.ctypes.data_as(u32p), limbs_per_coeff))
    return limbs_to_ints(out)


class Strip:
    """A strip of width L (cp_create_strip / cp_advance_rows / cp_read_coeffs / cp_destroy).

    With ``v`` given, the any-v Potts strip (cp_create_strip_potts): the
    residues of Z~(w) = q^{-|V|} Z(q, v) instead of the chromatic P~.
    """

    def __init__(self, lattice, L, primes, max_degree=-1, max_rows=1, stream=None, v=None):
        pr, pp = _u32(primes)
        self.primes = [int(p) for p in pr]
        h = vp()
        s = stream if stream is None or isinstance(stream, int) else stream.cuda_stream
        sh = vp(s) if s else None
        if v is None:
            check("cp_create_strip", load().cp_create_strip(lattice_id(lattice), L, pp, len(pr), max_degree,
                                                            max_rows, sh, ctypes.byref(h)))
        else:
            check("cp_create_strip_potts", load().cp_create_strip_potts(lattice_id(lattice), L, int(v), pp, len(pr),
                                                                        max_degree, max_rows, sh, ctypes.byref(h)))
        self.v = v
        self._h = h
        ns = (ctypes.c_uint64 * 2)()
        deg, hgt = ctypes.c_int(), ctypes.c_int()
        check("cp_strip_info", load().cp_strip_info(h, ns, ctypes.byref(deg), ctypes.byref(hgt)))
        self.n_states = (int(ns[0]), int(ns[1]))
        self.degree = deg.value
        self.L = L

    @property
    def height(self):
        deg, hgt = ctypes.c_int(), ctypes.c_int()
        check("cp_strip_info", load().cp_strip_info(self._h, None, ctypes.byref(deg), ctypes.byref(hgt)))
        return hgt.value

    def advance(self, n_rows):
        check("cp_advance_rows", load().cp_advance_rows(self._h, n_rows))

    def read(self):
        out = np.zeros((len(self.primes), self.degree + 1), dtype=np.uint32)
        h = ctypes.c_int()
        check("cp_read_coeffs", load().cp_read_coeffs(self._h, out.ctypes.data_as(u32p), out.size, ctypes.byref(h)))
        return out

    def read_integers(self, limbs_per_coeff=None, strict=True):
        """Exact integer coefficients c_0..c_D of P~ (cp_read_integers): read-out, CRT and
        the sufficiency checks on the GPU.  strict: raise CPError(CP_EPRIMES) when the
        primes are too few; else return (integers, flags, status)."""
        lpc = limbs_per_coeff or limbs_for(len(self.primes))
        out = np.zeros((self.degree + 1, lpc), dtype=np.uint32)
        flags = np.zeros(self.degree + 1, dtype=np.uint32)
        h = ctypes.c_int()
        rc = load().cp_read_integers(self._h, out.ctypes.data_as(u32p), out.size, lpc, flags.ctypes.data_as(u32p),
                                     ctypes.byref(h))
        if strict or rc not in (0, CP_EPRIMES):
            check("cp_read_integers", rc)
            return limbs_to_ints(out)
        return limbs_to_ints(out), [int(f) for f in flags], rc

    def reset(self):
        check("cp_strip_reset", load().cp_strip_reset(self._h))

    def set_tile(self, tile):
        """Gather tile of this strip's launches (cp_strip_set_tile; 0 = default)."""
        check("cp_strip_set_tile", load().cp_strip_set_tile(self._h, int(tile)))

    def work(self):
        """(row updates, row bytes, read-out updates, read-out bytes, row bytes one factor at a
        time, read-out bytes one factor at a time); see cp_strip_work."""
        w = (ctypes.c_uint64 * 6)()
        check("cp_strip_work", load().cp_strip_work(self._h, w))
        return tuple(int(x) for x in w)

    def read_device(self, ptr, n_words):
        check("cp_read_coeffs_device", load().cp_read_coeffs_device(self._h, vp(ptr), n_words))

    def close(self):
        if self._h:
            load().cp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def set_factor_pairing(mode):
    """Layout of square-lattice tables built from now on (cp_set_factor_pairing): 0 one
    table per site factor, 1 two-site tables for rows of at least 3 KB (default), 2
    two-site tables always.  Returns the previous mode."""
    return int(load().cp_set_factor_pairing(int(mode)))


def debug_check_space(kind, m, e=0):
    bad, size = ctypes.c_uint64(), ctypes.c_uint64()
    check("cp_debug_check_space", load().cp_debug_check_space(kind, m, e, ctypes.byref(bad), ctypes.byref(size)))
    return int(bad.value), int(size.value)


def debug_reduce(values, primes):
    """The gather kernels' modular reduction on the GPU: [v mod p for v, p in zip(values, primes)]."""
    v = np.ascontiguousarray(np.asarray(values, dtype=np.int64))
    p, pp = _u32(primes)
    out = np.zeros(len(v), dtype=np.uint32)
    check("cp_debug_reduce", load().cp_debug_reduce(v.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), pp, len(v),
                                                    out.ctypes.data_as(u32p)))
    return [int(x) for x in out]


def debug_reduce_halves(lo, hi, primes, full=True):
    """The bulk-copy gather's 32-bit reduction of u = hi 2^16 + lo on the GPU
    (cp_debug_reduce_halves): u mod p, or a representative in [-p, p) (as
    signed ints) when full is False."""
    lo_a = np.ascontiguousarray(np.asarray(lo, dtype=np.int32))
    hi_a = np.ascontiguousarray(np.asarray(hi, dtype=np.int32))
    p, pp = _u32(primes)
    out = np.zeros(len(lo_a), dtype=np.uint32)
    i32p = ctypes.POINTER(ctypes.c_int32)
    check("cp_debug_reduce_halves", load().cp_debug_reduce_halves(lo_a.ctypes.data_as(i32p), hi_a.ctypes.data_as(i32p),
                                                                  pp, len(lo_a), 1 if full else 0,
                                                                  out.ctypes.data_as(u32p)))
    return [int(x) for x in (out if full else out.view(np.int32))]


def debug_table(lattice, L, paired, which, index):
    """(row_ptr, edges, (n_src, n_dst, nnz, src_bits)) of one table (cp_debug_table)."""
    info = (ctypes.c_uint64 * 4)()
    check("cp_debug_table", load().cp_debug_table(lattice_id(lattice), L, paired, which, index, None, 0, None, 0,
                                                  info))
    n_src, n_dst, nnz, sb = (int(x) for x in info)
    rp = np.zeros(n_dst + 1, dtype=np.uint32)
    ed = np.zeros(max(nnz, 1), dtype=np.uint32)
    check("cp_debug_table", load().cp_debug_table(lattice_id(lattice), L, paired, which, index,
                                                  rp.ctypes.data_as(u32p), rp.size, ed.ctypes.data_as(u32p), ed.size,
                                                  info))
    return rp, ed[:nnz], (n_src, n_dst, nnz, sb)


def debug_enumerate_space(kind, m, e=0, max_states=1 << 22):
    buf = np.zeros(max_states * m, dtype=np.uint8)
    size = ctypes.c_uint64()
    check("cp_debug_enumerate_space", load().cp_debug_enumerate_space(
        kind, m, e, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), max_states, ctypes.byref(size)))
    return buf[: int(size.value) * m].reshape(int(size.value), m)


def _stream_handle(stream):
    if stream is None:
        return None
    return stream if isinstance(stream, int) else stream.cuda_stream


class Sweep:
    """The batched finite-lattice sweep (cp_sweep_*): all band rectangles of
    order k on the given primes, advanced together in one graph launch."""

    def __init__(self, lattice, k, primes, stream, tile=0, prime_groups=0):
        pr, pp = _u32(primes)
        self.primes = [int(p) for p in pr]
        self.lattice = lattice
        self.k = k
        h = vp()
        check("cp_sweep_create", load().cp_sweep_create(lattice_id(lattice), k, pp, len(pr), tile, prime_groups,
                                                        vp(_stream_handle(stream)), ctypes.byref(h)))
        self._h = h
        vals = [ctypes.c_int() for _ in range(4)] + [ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int()]
        check("cp_sweep_info", load().cp_sweep_info(h, *[ctypes.byref(v) for v in vals]))
        (self.n_rects, self.n_terms, self.tile, self.prime_groups, self.updates_per_run, self.bytes_per_run,
         self.launches_per_run) = [v.value for v in vals]
        w = (ctypes.c_uint64 * 3)()
        check("cp_sweep_work", load().cp_sweep_work(h, w))
        self.site_bytes_per_run = int(w[2])  # the same work one factor at a time
        rs = (ctypes.c_int * (2 * self.n_rects))()
        check("cp_sweep_rects", load().cp_sweep_rects(h, rs, self.n_rects))
        self.rects = [(rs[2 * j], rs[2 * j + 1]) for j in range(self.n_rects)]

    def run(self):
        check("cp_sweep_run", load().cp_sweep_run(self._h))

    def sync(self):
        check("cp_sweep_sync", load().cp_sweep_sync(self._h))

    def read_ptilde(self):
        """{(r, s): uint32 [n_primes][n_terms]}"""
        out = np.zeros((self.n_rects, len(self.primes), self.n_terms), dtype=np.uint32)
        check("cp_sweep_read_ptilde", load().cp_sweep_read_ptilde(self._h, out.ctypes.data_as(u32p), out.size))
        return {rs: out[j] for j, rs in enumerate(self.rects)}

    def read_series(self):
        """uint32 [3][n_primes][n_terms]: bulk, surface, corner residues."""
        out = np.zeros((3, len(self.primes), self.n_terms), dtype=np.uint32)
        check("cp_sweep_read_series", load().cp_sweep_read_series(self._h, out.ctypes.data_as(u32p), out.size))
        return out

    def set_primes(self, primes):
        pr, pp = _u32(primes)
        check("cp_sweep_set_primes", load().cp_sweep_set_primes(self._h, pp, len(pr)))
        self.primes = [int(p) for p in pr]

    def profile(self):
        """(summed gather kernel ms, gather launches, whole pass ms) of one ungraphed pass."""
        g, n, t = ctypes.c_float(), ctypes.c_int(), ctypes.c_float()
        check("cp_sweep_profile", load().cp_sweep_profile(self._h, ctypes.byref(g), ctypes.byref(n), ctypes.byref(t)))
        return g.value, n.value, t.value

    def read_series_device(self, ptr, n_words):
        check("cp_sweep_read_series_device", load().cp_sweep_read_series_device(self._h, vp(ptr), n_words))

    def series_integers(self, limbs_per_coeff=None, out=None):
        """The three series as exact integers, CRT'd and checked for stability on the GPU
        (cp_sweep_series_integers); raises CPError(CP_EPRIMES) if a term is not stable.
        out: optional uint32 array [3][n_terms][limbs] (e.g. pinned) to receive the limbs."""
        lpc = limbs_per_coeff or limbs_for(len(self.primes))
        if out is None:
            out = np.zeros((3, self.n_terms, lpc), dtype=np.uint32)
        check("cp_sweep_series_integers", load().cp_sweep_series_integers(
            self._h, out.ctypes.data_as(u32p), out.size, lpc, None))
        return [limbs_to_ints(out[x]) for x in range(3)]

    def close(self):
        if self._h:
            load().cp_sweep_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching server of rectangle solves (cp_server_*)."""

    QUEUED, ACTIVE, DONE, FAILED = 0, 1, 2, -1

    def __init__(self, mem_budget_bytes, max_active=64, stream=None):
        h = vp()
        check("cp_server_create", load().cp_server_create(int(mem_budget_bytes), int(max_active),
                                                          vp(_stream_handle(stream)), ctypes.byref(h)))
        self._h = h
        self.shapes = {}

    def submit(self, lattice, L, N, primes):
        pr, pp = _u32(primes)
        rid = ctypes.c_uint64()
        check("cp_server_submit", load().cp_server_submit(self._h, lattice_id(lattice), L, N, pp, len(pr),
                                                          ctypes.byref(rid)))
        self.shapes[rid.value] = (len(pr), L * N)
        return rid.value

    def step(self):
        a, q, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check("cp_server_step", load().cp_server_step(self._h, ctypes.byref(a), ctypes.byref(q), ctypes.byref(f)))
        return a.value, q.value, f.value

    def result(self, rid):
        """(state, residues [P][L*N] or None, (t_submit, t_admit, t_done))"""
        P, n = self.shapes[rid]
        out = np.zeros((P, n), dtype=np.uint32)
        st = ctypes.c_int()
        ts = (ctypes.c_double * 3)()
        check("cp_server_result", load().cp_server_result(self._h, rid, out.ctypes.data_as(u32p), out.size,
                                                          ctypes.byref(st), ts))
        return st.value, (out if st.value == self.DONE else None), tuple(ts)

    def poll(self, max_ids=4096):
        """Ids finished since the last poll."""
        buf = (ctypes.c_uint64 * max_ids)()
        n = ctypes.c_int()
        check("cp_server_poll", load().cp_server_poll(self._h, buf, max_ids, ctypes.byref(n)))
        return [int(buf[k]) for k in range(n.value)]

    def cancel(self, rid):
        check("cp_server_cancel", load().cp_server_cancel(self._h, rid))

    def release(self, rid):
        check("cp_server_release", load().cp_server_release(self._h, rid))
        self.shapes.pop(rid, None)

    def stats(self):
        s, l, u, f = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_size_t()
        check("cp_server_stats", load().cp_server_stats(self._h, ctypes.byref(s), ctypes.byref(l), ctypes.byref(u),
                                                        ctypes.byref(f)))
        return {"steps": s.value, "launches": l.value, "updates": u.value, "arena_free_bytes": f.value}

    def close(self):
        if self._h:
            load().cp_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
