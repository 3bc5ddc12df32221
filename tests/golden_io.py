"""Readers for the fixtures under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                yield ln.split()


def ptilde(lattice, L, N):
    return [int(r[1]) for r in _rows("ptilde_%s_%dx%d.txt" % (lattice, L, N))]


def table1():
    """{'alpha': [...], 'beta': [...], 'gamma': [...]} from Table 1 (Sec. 4.2)."""
    a, b, g = [], [], []
    for r in _rows("table1_square.txt"):
        a.append(int(r[1]))
        b.append(int(r[2]))
        if r[3] != "-":
            g.append(int(r[3]))
    return {"alpha": a, "beta": b, "gamma": g}


def triangular_series():
    """{'surface': [...], 'corner': [...]} x^0..x^40, eqs. (efs_ser), (efc_ser)."""
    s, c = [], []
    for r in _rows("triangular_series.txt"):
        s.append(int(r[1]))
        c.append(int(r[2]))
    return {"surface": s, "corner": c}
