"""Connectivity states: set partitions of the m top-row sites (Sec. 3, 3.2, 3.4).

Test infrastructure only (see ``oracle/__init__``).

A partition of the sites 0..m-1 (the paper's 1..m) is stored as a tuple of
block labels in first-occurrence order, e.g. (0, 1, 0, 2) is (13)(2)(4).

* non-crossing: no a < b < c < d with a~c, b~d and a !~ b (Sec. 3.2);
* NCNNN: non-crossing and no two neighbouring sites in one block (Sec. 3.2);
  the square-lattice intermediate spaces lift the neighbour rule on one pair
  (i, i+1) (Sec. 3.4, last paragraph).

Counts: Catalan C_m and Motzkin M_k by the paper's closed sums (Sec. 3.2).

The paper's ordering of the NCNNN partitions (Sec. 3.4) is generated here
literally from its recursive description: first the partitions where point 1
is alone (ordered as the partitions of points 2..m), then, for increasing k,
those where 3+k is the smallest partner of 1, ordered by the partition of the
inner points 2..2+k (most significant) and then by that of the right points
3+k..m (least significant).  Ranks are 0-based positions in that list (the
paper counts from 1); the rank maps here are plain dictionaries.
"""
from functools import lru_cache
from math import comb, factorial


def canon(labels):
    """Relabel blocks in first-occurrence order."""
    seen = {}
    out = []
    for x in labels:
        if x not in seen:
            seen[x] = len(seen)
        out.append(seen[x])
    return tuple(out)


def from_blocks(m, blocks):
    lab = [None] * m
    for b, blk in enumerate(blocks):
        for p in blk:
            lab[p] = b
    assert None not in lab
    return canon(lab)


def to_str(s):
    """Paper notation with 1-based points, blocks ordered by first point."""
    blocks = {}
    for p, b in enumerate(s):
        blocks.setdefault(b, []).append(p + 1)
    return "".join("(" + "".join(str(p) for p in blk) + ")" for blk in blocks.values())


def is_noncrossing(s):
    m = len(s)
    for a in range(m):
        for b in range(a + 1, m):
            if s[b] == s[a]:
                continue
            for c in range(b + 1, m):
                if s[c] != s[a]:
                    continue
                for d in range(c + 1, m):
                    if s[d] == s[b]:
                        return False
    return True


def nn_ok(s, skip=None):
    """No neighbouring pair (j, j+1) in one block, except the pair j == skip."""
    return all(s[j] != s[j + 1] for j in range(len(s) - 1) if j != skip)


def catalan(m):
    return factorial(2 * m) // (factorial(m) * factorial(m + 1))


def motzkin(k):
    return sum(comb(k, 2 * j) * catalan(j) for j in range(k // 2 + 1))


def all_partitions(m):
    """Every set partition of m points (restricted growth strings)."""
    out = []

    def rec(prefix, nb):
        if len(prefix) == m:
            out.append(tuple(prefix))
            return
        for b in range(nb + 1):
            rec(prefix + [b], max(nb, b + 1))

    rec([], 0)
    return out


@lru_cache(maxsize=None)
def _ordered_blocks(lo, hi):
    """NCNNN partitions of points lo..hi-1 in the paper's order, as block lists."""
    n = hi - lo
    if n == 0:
        return ((),)
    if n == 1:
        return (((lo,),),)
    res = []
    # (i) point lo alone; rest ordered as the partitions of lo+1..hi-1
    for rest in _ordered_blocks(lo + 1, hi):
        res.append(((lo,),) + rest)
    # (ii) smallest partner of lo is lo+2+k, k = 0..n-3
    for k in range(n - 2):
        partner = lo + 2 + k
        for inner in _ordered_blocks(lo + 1, partner):      # most significant
            for right in _ordered_blocks(partner, hi):      # least significant
                blocks = list(inner)
                for blk in right:
                    blocks.append(((lo,) + blk) if partner in blk else blk)
                res.append(tuple(blocks))
    return tuple(res)


@lru_cache(maxsize=None)
def ncnnn_ordered(m):
    """The M_{m-1} NCNNN partitions of m points in the paper's order (Sec. 3.4)."""
    return tuple(from_blocks(m, b) for b in _ordered_blocks(0, m))


@lru_cache(maxsize=None)
def excepted_ordered(m, e):
    """Square-lattice intermediate space where only the pair (e, e+1) may share
    a block: the NCNNN partitions first, then the partitions with e ~ e+1 in the
    order of their contraction to m-1 points (Sec. 3.4, last paragraph)."""
    out = list(ncnnn_ordered(m))
    for c in ncnnn_ordered(m - 1):
        lab = list(c[: e + 1]) + [c[e]] + list(c[e + 1:])
        out.append(canon(lab))
    return tuple(out)


@lru_cache(maxsize=None)
def rank_map(space):
    """space = ('B', m) or ('X', m, e): dict partition -> 0-based rank."""
    if space[0] == "B":
        lst = ncnnn_ordered(space[1])
    else:
        lst = excepted_ordered(space[1], space[2])
    return {s: r for r, s in enumerate(lst)}


def space_list(space):
    if space[0] == "B":
        return ncnnn_ordered(space[1])
    return excepted_ordered(space[1], space[2])
