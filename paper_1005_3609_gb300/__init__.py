"""GB300-native sparse transfer matrix for the chromatic polynomial (arXiv:1005.3609).

The computation lives in the CUDA library libcp_gb300.so (C ABI in
include/cp_tm.h); this package is its Python binding.  Importing it does not
load the library; the first call does, and raises if it is not built.
"""
from ._lib import (CP_EPRIMES, CP_MAX_L, CP_MAX_PRIMES, CPError, Server, Strip, Sweep, crt, crt_checked,  # noqa: F401
                   crt_static, debug_check_space, debug_enumerate_space, load, select_primes, set_factor_pairing,
                   whitney_bits)
