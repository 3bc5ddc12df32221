"""Paper-scale finite-lattice sweeps, k = 41 (widths up to 20, the paper's m_max; Sec. 4.2, 4.3).

The square sweep reproduces all of Table 1: alpha_k and beta_k for k = 0..79 (z^79 through
the mu_40 term) and gamma_k for k = 0..78.  The triangular sweep reproduces Baxter's
product, eq. (efb), the printed series (efs_ser), (efc_ser) and the conjectured product
formulae (efs), (efc) through x^40.
Four primes suffice (the largest coefficient, |gamma_78|, is below 2^88).  The square sweep
holds ~120 GB of state vectors on the device (the width-20 intermediate space has
M_19 + M_18 = 24 735 666 states).
"""
import pytest

import golden_io
import gpu_util
from oracle import flm

pytestmark = pytest.mark.gpu

cp = pytest.importorskip("paper_1005_3609_gb300")

TILE = 32  # TMA gather, 32 rows per block, stages and chunks per thread picked from the row width (no autotune at this size)


@pytest.fixture(scope="module")
def stream():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cp.load()
    return torch.cuda.Stream()


def test_square_k41_reproduces_table1(stream):
    primes = gpu_util.seed_primes(4)
    t = golden_io.table1()
    with cp.Sweep("square", 41, primes, stream, tile=TILE, prime_groups=1) as sw:
        assert sw.n_terms == 80 and max(r for r, _ in sw.rects) == 20
        sw.run()
        sw.sync()
        bulk, surf, corner = sw.series_integers()
    assert bulk == t["alpha"]          # z^0..z^79
    assert surf == t["beta"]           # z^0..z^79
    assert corner[:79] == t["gamma"]   # z^0..z^78
    cp.load().cp_clear_table_cache()


def test_triangular_k41_reproduces_baxter_and_printed(stream):
    primes = gpu_util.seed_primes(4)
    tri = golden_io.triangular_series()
    with cp.Sweep("triangular", 41, primes, stream, tile=TILE, prime_groups=1) as sw:
        assert sw.n_terms == 41
        sw.run()
        sw.sync()
        bulk, surf, corner = sw.series_integers()
    assert bulk == flm.baxter_bulk(41)
    assert surf == tri["surface"]
    assert corner == tri["corner"]
    # the conjectured product formulae, eqs. (efs) and (efc), through x^40
    assert surf == flm.conjectured_surface(41)
    assert corner == flm.conjectured_corner(41)
    cp.load().cp_clear_table_cache()
