"""Pins of the oracle's finite-lattice method against Table 1, Baxter and the printed series (Sec. 4)."""
import pytest

import golden_io
import synthetic_inputs
from oracle import crt, flm, modp, tm_exact


@pytest.mark.parametrize("k", [8, 13, 20, 33, 41])
def test_sum_rules(k):
    B = flm.band(k)
    moments = lambda f: (sum(f(k, r, s) * r * s for r, s in B), sum(f(k, r, s) * (r + s) for r, s in B),
                         sum(f(k, r, s) for r, s in B))
    assert moments(flm.alpha) == (1, 0, 0)
    assert moments(flm.beta) == (0, 1, 0)
    assert moments(flm.gamma) == (0, 0, 1)
    assert moments(flm.beta_printed) != (0, 1, 0)  # the printed (r+s-2)/2 fails


def test_band_size():
    assert len(flm.band(33)) == 62
    assert max(r for r, _ in flm.band(33)) == 16


def _ptildes_exact(lattice, k, D):
    out = {}
    for r in range(1, k // 2 + 1):
        hs = [s for rr, s in flm.band(k) if rr == r]
        got = tm_exact.ptilde_heights(lattice, r, hs, D)
        out.update({(r, s): got[s] for s in hs})
    return out


def test_table1_k17_exact_with_mu_term():
    # k = 17, m_max = 8: series exact through z^30, and the mu_16 z^31 term of Sec. 4.2 gives z^31
    k, mmax = 17, 8
    n = flm.n_terms("square", k) + 1
    a, b, g = flm.flm_series("square", k, _ptildes_exact("square", k, n - 1), n)
    t = golden_io.table1()
    assert a[: n - 1] == t["alpha"][: n - 1]
    assert b[: n - 1] == t["beta"][: n - 1]
    assert g[: n - 1] == t["gamma"][: n - 1]
    mu = flm.mu_series(2 * mmax)
    assert a[n - 1] + mu[2 * mmax] == t["alpha"][n - 1]
    assert b[n - 1] - mmax * mu[2 * mmax] == t["beta"][n - 1]


def test_table1_k21_modp_crt():
    # through the plain-C mod-p oracle and CRT: z^0..z^38 and the mu_20 z^39 term
    k, mmax = 21, 10
    n = flm.n_terms("square", k) + 1
    primes = crt.primes_from_draws(synthetic_inputs.prime_draws(0, 32), 3)
    per_prime = []
    for p in primes:
        pt = {}
        for r in range(1, mmax + 1):
            hs = [s for rr, s in flm.band(k) if rr == r]
            got = modp.ptilde_heights("square", r, hs, n - 1, p)
            pt.update({(r, s): [int(x) for x in got[s]] for s in hs})
        a, b, g = flm.flm_series("square", k, pt, n)
        per_prime.append(([x % p for x in a], [x % p for x in b], [x % p for x in g]))
    t = golden_io.table1()
    for idx, name in enumerate(["alpha", "beta", "gamma"]):
        got = crt.crt_signed([pp[idx] for pp in per_prime], primes)
        assert got[: n - 1] == t[name][: n - 1], name
    mu = flm.mu_series(2 * mmax)
    a = crt.crt_signed([pp[0] for pp in per_prime], primes)
    b = crt.crt_signed([pp[1] for pp in per_prime], primes)
    assert a[n - 1] + mu[2 * mmax] == t["alpha"][n - 1]
    assert b[n - 1] - mmax * mu[2 * mmax] == t["beta"][n - 1]


def test_triangular_k13_against_baxter_and_printed():
    k = 13
    n = flm.n_terms("triangular", k)
    bulk, surf, corn = flm.flm_series("triangular", k, _ptildes_exact("triangular", k, n - 1), n)
    tri = golden_io.triangular_series()
    assert bulk == flm.baxter_bulk(n)
    assert surf == tri["surface"][:n]
    assert corn == tri["corner"][:n]


def test_baxter_first_terms():
    assert flm.baxter_bulk(16) == [1, 1, 2, 1, 0, -2, -2, 0, 3, 5, 2, -4, -10, -8, 3, 15]


def test_conjectured_products_reproduce_printed_series():
    # eqs. (efs), (efc) against eqs. (efs_ser), (efc_ser) through x^40
    tri = golden_io.triangular_series()
    assert flm.conjectured_surface(41) == tri["surface"]
    assert flm.conjectured_corner(41) == tri["corner"]


def test_mu_integral():
    mu = flm.mu_series(40)
    assert mu[:4] == [0, 0, 0, 0]
    assert all(isinstance(x, int) and x > 0 for x in mu[4:])


def test_series_ops():
    n = 12
    a = [1, 3, -2, 5] + [0] * 8
    assert flm.mul(a, flm.inverse(a, n), n) == [1] + [0] * (n - 1)
    assert flm.power(a, 3, n) == flm.mul(a, flm.mul(a, a, n), n)
    assert flm.mul(flm.power(a, -2, n), flm.power(a, 2, n), n) == [1] + [0] * (n - 1)
    # w(z) = z/(1+z) inverts z = w/(1-w)
    w = flm.w_of_z(n)
    z_of_w = [0] + [1] * (n - 1)
    assert flm.compose_w(z_of_w, w, n) == [0, 1] + [0] * (n - 2)
