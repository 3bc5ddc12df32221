"""The plain any-v transfer matrix on non-crossing partitions (Sec. 3.1-3.2).

Test infrastructure only (see ``oracle/__init__``).

This is the construction T = (prod_i V_i)(prod_i H_{i,i+1}) that the paper
improves on: no projector, no non-nearest-neighbour restriction, any v.  It is
an independent check of the projected factorisation in ``tm_exact``: it uses
its own state representation (a frozenset of frozenset blocks) and its own
operator code.

Triangular lattice: after the horizontal edges of a layer, site i is moved up
(V_i) and then the diagonal joins the moved site i to the not-yet-moved site
i+1 (new (t+1, i) to old (t, i+1)), the orientation of Sec. 3.3.

After the last layer's horizontal edges every remaining block is a finished
component whose q and w factors are already counted, so Z~ is the sum of all
state weights.
"""


def _norm(blocks):
    return frozenset(frozenset(b) for b in blocks)


def _join(state, a, b):
    ba = next(x for x in state if a in x)
    bb = next(x for x in state if b in x)
    if ba == bb:
        return state, 0
    return _norm([x for x in state if x not in (ba, bb)] + [ba | bb]), 1


def _detach(state, i):
    bi = next(x for x in state if i in x)
    rest = [x for x in state if x != bi]
    if len(bi) > 1:
        rest.append(bi - {i})
    rest.append(frozenset({i}))
    return _norm(rest)


def _add(out, st, poly, coef, shift, deg):
    tgt = out.setdefault(st, [0] * (deg + 1))
    for j in range(deg + 1 - shift):
        tgt[j + shift] += coef * poly[j]


def _H(vec, a, b, v, deg):
    out = {}
    for st, p in vec.items():
        _add(out, st, p, 1, 0, deg)
        t, k = _join(st, a, b)
        _add(out, t, p, v, k, deg)
    return out


def _V(vec, i, v, deg):
    out = {}
    for st, p in vec.items():
        _add(out, _detach(st, i), p, 1, 0, deg)
        _add(out, st, p, v, 1, deg)
    return out


def ztilde(lattice, L, N, v):
    """Coefficients of Z~(w) = q^{-LN} Z(q, v) for the L x N rectangle."""
    deg = L * N - 1
    vec = {_norm([[i] for i in range(L)]): [1] + [0] * deg}
    for _ in range(N - 1):
        for i in range(L - 1):
            vec = _H(vec, i, i + 1, v, deg)
        for i in range(L):
            vec = _V(vec, i, v, deg)
            if lattice == "triangular" and i + 1 < L:
                vec = _H(vec, i, i + 1, v, deg)
    for i in range(L - 1):
        vec = _H(vec, i, i + 1, v, deg)
    total = [0] * (deg + 1)
    for p in vec.values():
        for j in range(deg + 1):
            total[j] += p[j]
    return total


def reachable_states(L, n_rows, lattice="square"):
    """Partitions reached by the any-v matrix (all non-crossing ones for v != 0)."""
    vec = {_norm([[i] for i in range(L)]): [1]}
    seen = set(vec)
    for _ in range(n_rows):
        for i in range(L - 1):
            vec = _H(vec, i, i + 1, 1, 0)
            seen |= set(vec)
        for i in range(L):
            vec = _V(vec, i, 1, 0)
            seen |= set(vec)
    return seen
