"""Pins of the oracle's transfer matrices against definitions, closed forms and invariants."""
from math import comb

import pytest

import golden_io
import synthetic_inputs
from oracle import brute, crt, delcon, fk, graphs, modp, tm_exact, tm_generic

TINY = [(1, 1), (1, 4), (2, 1), (2, 2), (2, 3), (3, 2), (3, 3), (2, 5), (4, 2), (3, 4), (4, 3)]


def ptilde_from_q(coeffs_q, nv):
    """P(q) ascending in q -> P~ ascending in w = 1/q."""
    return [coeffs_q[nv - j] for j in range(nv)]


def expand_q_poly(factors, nv):
    """Product of polynomials in q (ascending lists) -> P~ coefficients."""
    out = [1]
    for f in factors:
        nxt = [0] * (len(out) + len(f) - 1)
        for i, a in enumerate(out):
            for j, b in enumerate(f):
                nxt[i + j] += a * b
        out = nxt
    out += [0] * (nv + 1 - len(out))
    return ptilde_from_q(out, nv)


@pytest.mark.parametrize("lattice", ["square", "triangular"])
@pytest.mark.parametrize("L,N", TINY)
def test_against_colourings_and_deletion_contraction(lattice, L, N):
    nv, edges = graphs.rectangle_edges(lattice, L, N)
    want = ptilde_from_q(brute.chromatic_poly(lattice, L, N), nv)
    assert ptilde_from_q(delcon.chromatic_poly(nv, edges), nv) == want
    assert tm_exact.ptilde(lattice, L, N) == want
    assert tm_generic.ztilde(lattice, L, N, -1) == want
    if len(edges) <= 16:
        assert fk.ztilde(nv, edges, -1) == want


@pytest.mark.parametrize("lattice", ["square", "triangular"])
@pytest.mark.parametrize("v", [2, 3, -2])
def test_generic_v_against_fk(lattice, v):
    for L, N in [(2, 2), (3, 2), (2, 3), (3, 3)]:
        nv, edges = graphs.rectangle_edges(lattice, L, N)
        if len(edges) > 16:
            continue
        assert tm_generic.ztilde(lattice, L, N, v) == fk.ztilde(nv, edges, v)


def test_hand_trace_m2_n2():
    # e0 -T_1-> (1-2w) e0 + w^2 (12) -T_2-> (1-3w+3w^2) e0 -T_last-> 1-4w+6w^2-3w^3
    D = 3
    v = tm_exact.e0(2, D)
    v = tm_exact.site_op("square", 2, 0, v, D)
    assert v == {(0, 1): [1, -2, 0, 0], (0, 0): [0, 0, 1, 0]}
    v = tm_exact.site_op("square", 2, 1, v, D)
    assert v == {(0, 1): [1, -3, 3, 0]}
    assert tm_exact.readout(2, v, D) == [1, -4, 6, -3]


@pytest.mark.parametrize("N", range(1, 12))
def test_width_one(N):
    want = [(-1) ** j * comb(N - 1, j) for j in range(N)]  # (1-w)^{N-1}
    assert tm_exact.ptilde("square", 1, N) == want
    assert tm_exact.ptilde("triangular", 1, N) == want
    assert tm_exact.ptilde("square", N, 1) == want


@pytest.mark.parametrize("N", range(1, 21))
def test_two_by_n_square_closed_form(N):
    want = expand_q_poly([[0, 1], [-1, 1]] + [[3, -3, 1]] * (N - 1), 2 * N)
    assert tm_exact.ptilde("square", 2, N) == want


@pytest.mark.parametrize("N", range(2, 41))
def test_two_by_n_triangular_closed_form(N):
    want = expand_q_poly([[0, 1], [-1, 1]] + [[-2, 1]] * (2 * N - 2), 2 * N)
    assert tm_exact.ptilde("triangular", 2, N) == want


def check_invariants(lattice, L, N, c):
    nv, edges = graphs.rectangle_edges(lattice, L, N)
    E = len(edges)
    assert len(c) == nv
    assert c[0] == 1
    assert c[1] == -E
    if nv > 2:
        assert c[2] == comb(E, 2) - graphs.count_triangles(nv, edges)
    assert all((-1) ** j * c[j] > 0 for j in range(nv))     # connected graph
    assert all(abs(c[j]) <= comb(E, j) for j in range(nv))    # Whitney's broken circuits
    assert sum(c) == 0                                         # P(1) = 0
    p2 = sum(cj * 2 ** (nv - j) for j, cj in enumerate(c))
    p3 = sum(cj * 3 ** (nv - j) for j, cj in enumerate(c))
    if L >= 2 and N >= 2:
        if lattice == "square":
            assert p2 == 2                                     # connected bipartite
        else:
            assert p2 == 0 and p3 == 6                         # triangulated disc


@pytest.mark.parametrize("lattice", ["square", "triangular"])
@pytest.mark.parametrize("L,N", [(3, 5), (4, 4), (5, 3), (4, 6), (5, 5)])
def test_invariants_and_transpose(lattice, L, N):
    a = tm_exact.ptilde(lattice, L, N)
    check_invariants(lattice, L, N, a)
    assert tm_exact.ptilde(lattice, N, L) == a


def test_golden_config1_matches_exact():
    assert golden_io.ptilde("square", 5, 6) == tm_exact.ptilde("square", 5, 6)
    check_invariants("square", 5, 6, golden_io.ptilde("square", 5, 6))


@pytest.mark.parametrize("lattice,L,N", [("square", 12, 13), ("triangular", 13, 14)])
def test_golden_large_invariants(lattice, L, N):
    check_invariants(lattice, L, N, golden_io.ptilde(lattice, L, N))


def test_golden_square_12x13_one_fresh_prime():
    # a prime that the golden CRT did not use
    p = crt.primes_from_draws(synthetic_inputs.prime_draws(12345, 8), 1)[0]
    want = [c % p for c in golden_io.ptilde("square", 12, 13)]
    assert [int(x) for x in modp.ptilde("square", 12, 13, 155, p)] == want


@pytest.mark.parametrize("lattice", ["square", "triangular"])
def test_modp_matches_exact(lattice):
    primes = crt.primes_from_draws(synthetic_inputs.prime_draws(0, 16), 3) + [2147483647, 3]
    for L, N, D in [(1, 1, 0), (1, 5, 4), (3, 4, 11), (5, 6, 29), (6, 5, 7), (7, 3, 20), (4, 7, 0)]:
        ex = tm_exact.ptilde(lattice, L, N, D)
        for p in primes:
            assert [int(x) for x in modp.ptilde(lattice, L, N, D, p)] == [c % p for c in ex]


def test_modp_transpose_medium():
    p = 2147483647
    for lattice in ("square", "triangular"):
        a = modp.ptilde(lattice, 6, 9, 53, p)
        b = modp.ptilde(lattice, 9, 6, 53, p)
        assert list(a) == list(b)


def test_truncation_is_a_prefix():
    full = tm_exact.ptilde("triangular", 4, 5)
    for D in (0, 1, 5, 12):
        assert tm_exact.ptilde("triangular", 4, 5, D) == full[: D + 1]
