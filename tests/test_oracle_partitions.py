"""Pins of the oracle's state space: the paper's printed orderings and counts (Sec. 3.2-3.4)."""
import pytest

from oracle import partitions as P
from oracle import tm_generic


def test_m3_noncrossing_states():
    # Sec. 3: the five states for m = 3
    got = sorted(P.to_str(s) for s in P.all_partitions(3) if P.is_noncrossing(s))
    assert got == sorted(["(1)(2)(3)", "(12)(3)", "(13)(2)", "(1)(23)", "(123)"])


def test_m4_ncnnn_order():
    # Sec. 3.2, the four NCNNN partitions of m = 4 in the printed order
    assert [P.to_str(s) for s in P.ncnnn_ordered(4)] == ["(1)(2)(3)(4)", "(1)(24)(3)", "(13)(2)(4)", "(14)(2)(3)"]


def test_m5_ncnnn_order():
    # Sec. 3.4, the printed ordering of the nine NCNNN partitions of m = 5
    assert [P.to_str(s) for s in P.ncnnn_ordered(5)] == [
        "(1)(2)(3)(4)(5)", "(1)(2)(35)(4)", "(1)(24)(3)(5)", "(1)(25)(3)(4)",
        "(13)(2)(4)(5)", "(135)(2)(4)", "(14)(2)(3)(5)", "(15)(2)(3)(4)", "(15)(24)(3)"]


def test_counts_printed():
    # Sec. 3.2: C_m = 1,2,5,14,42,132 and M_k = 1,1,2,4,9,21
    assert [P.catalan(m) for m in range(1, 7)] == [1, 2, 5, 14, 42, 132]
    assert [P.motzkin(k) for k in range(6)] == [1, 1, 2, 4, 9, 21]


def test_motzkin_recursion_and_dimensions():
    # eq. (M_recurs) against the closed sum, and the dimensions of Sec. 4.2 / 4.3
    M = [1, 1]
    for p in range(2, 26):
        M.append(M[p - 1] + sum(M[k] * M[p - k - 2] for k in range(p - 1)))
    assert M == [P.motzkin(k) for k in range(26)]
    assert M[19] + M[18] == 24735666
    assert M[19] == 18199284


@pytest.mark.parametrize("m", range(1, 10))
def test_ncnnn_space_is_the_filtered_set(m):
    allp = P.all_partitions(m)
    want = {s for s in allp if P.is_noncrossing(s) and P.nn_ok(s)}
    got = P.ncnnn_ordered(m)
    assert len(got) == len(set(got)) == P.motzkin(m - 1)
    assert set(got) == want


@pytest.mark.parametrize("m", range(2, 9))
def test_excepted_spaces(m):
    # Sec. 3.4 last paragraph: M_{m-1} + M_{m-2} partitions, NCNNN ones first
    allp = P.all_partitions(m)
    for e in range(m - 1):
        lst = P.excepted_ordered(m, e)
        want = {s for s in allp if P.is_noncrossing(s) and P.nn_ok(s, skip=e)}
        assert len(lst) == len(set(lst)) == P.motzkin(m - 1) + P.motzkin(m - 2)
        assert set(lst) == want
        nb = P.motzkin(m - 1)
        assert all(s[e] != s[e + 1] for s in lst[:nb])
        assert all(s[e] == s[e + 1] for s in lst[nb:])


@pytest.mark.parametrize("m", range(1, 7))
def test_generic_matrix_reaches_all_noncrossing(m):
    # Sec. 3.2: generic v reaches the C_m non-crossing partitions
    assert len(tm_generic.reachable_states(m, m + 1)) == P.catalan(m)
