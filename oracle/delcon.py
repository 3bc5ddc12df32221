"""Chromatic polynomial by deletion-contraction (textbook recursion).

Test infrastructure only (see ``oracle/__init__``).

P(G) = P(G - e) - P(G / e) for any edge e, and P of the edgeless graph on n
vertices is q^n.  Parallel edges created by a contraction are merged (they do
not change P).  Memoised on the relabelled edge set.
"""
from functools import lru_cache


def _relabel(n, edges):
    used = sorted({x for e in edges for x in e})
    rank = {v: k for k, v in enumerate(used)}
    iso = n - len(used)  # isolated vertices each contribute a factor q
    return iso, len(used), frozenset((rank[u], rank[v]) for u, v in edges)


@lru_cache(maxsize=None)
def _p(n, edges):
    if not edges:
        out = [0] * (n + 1)
        out[n] = 1
        return tuple(out)
    e = min(edges)
    rest = edges - {e}
    a = _poly_of(n, rest)
    u, v = e
    contracted = set()
    for x, y in rest:
        x = u if x == v else x
        y = u if y == v else y
        if x == y:
            continue
        contracted.add((min(x, y), max(x, y)))
    b = _poly_of(n - 1, contracted)
    out = [0] * (n + 1)
    for k, c in enumerate(a):
        out[k] += c
    for k, c in enumerate(b):
        out[k] -= c
    return tuple(out)


def _poly_of(n, edges):
    iso, used, rel = _relabel(n, edges)
    inner = _p(used, rel)
    return [0] * iso + list(inner)


def chromatic_poly(n, edges):
    """Coefficients of P_G(q), ascending powers of q."""
    return _poly_of(n, frozenset((min(u, v), max(u, v)) for u, v in edges))
