"""Motion-vector probability statistics of Sec. II-C (the tables behind the
directional model, Sec. II-D), computed from the counts that me_mvp_stats
produces on the GPU.  Host arithmetic only: normalisation, folding, marginals,
regional sums, the statistic printed as eq. (1)-(2), and the conditional
distributions D1 (eq. (4)) and D2 (eq. (6)).

Conventions: a 2-D array P is indexed P[dy + R, dx + R]; Table II folds it to
|dy|, |dx|; Ax(d) = P(mv_x = d), Ay(d) = P(mv_y = d) (Table III, "accumulated
in the vertical / horizontal direction"), Bx(d) = P(mv = (d, 0)), By(d) =
P(mv = (0, d)).
"""
from __future__ import annotations

import numpy as np

# S1 of D1 in the order the counts use (the centre first, then the CDS first step)
S1 = [(0, 0), (-2, 0), (-1, 0), (1, 0), (2, 0), (0, 2), (0, 1), (0, -1), (0, -2)]
# S2 of D2: the 5x5 square, point i = (i % 5 - 2, i // 5 - 2)
S2 = [(i % 5 - 2, i // 5 - 2) for i in range(25)]


def unpack(counts, R):
    """Split the 35 * (2R+1)^2 counts of me_mvp_stats into (hist [side, side],
    d1 [9, side, side], d2 [side, side, 25]), side = 2R + 1."""
    side = 2 * R + 1
    q = side * side
    c = np.asarray(counts, dtype=np.int64).reshape(-1)
    assert c.size == 35 * q, "35 * (2R+1)^2 counts expected"
    hist = c[:q].reshape(side, side)
    d1 = c[q:10 * q].reshape(9, side, side)
    d2 = c[10 * q:].reshape(side, side, 25)
    return hist, d1, d2


def probabilities(hist):
    h = np.asarray(hist, dtype=np.float64)
    return h / max(h.sum(), 1.0)


def quarter_table(P):
    """Table II: P folded onto |dy| (rows) and |dx| (columns)."""
    side = P.shape[0]
    R = side // 2
    T = np.zeros((R + 1, R + 1))
    for iy in range(side):
        for ix in range(side):
            T[abs(iy - R), abs(ix - R)] += P[iy, ix]
    return T


def axes_1d(P):
    """Table III rows Ax, Ay, Bx, By over d = -R..R."""
    R = P.shape[0] // 2
    return {"Ax": P.sum(axis=0), "Ay": P.sum(axis=1), "Bx": P[R, :].copy(), "By": P[:, R].copy()}


def regions(P):
    """Regional probabilities of Fig. 3: the central 5x5 square (P), 5x5
    diamond, 5x5 cross, 3x3 square, and the flat region of the HCSP
    ((0,0), (+-1,0), (+-2,0), (0,+-1); printed 0.8248, Table VI's P1)."""
    R = P.shape[0] // 2

    def at(dx, dy):
        return P[dy + R, dx + R] if abs(dx) <= R and abs(dy) <= R else 0.0

    pts = [(dx, dy) for dy in range(-2, 3) for dx in range(-2, 3)]
    return {
        "square5": sum(at(x, y) for x, y in pts),
        "diamond5": sum(at(x, y) for x, y in pts if abs(x) + abs(y) <= 2),
        "cross5": sum(at(x, y) for x, y in pts if x == 0 or y == 0),
        "square3": sum(at(x, y) for x, y in pts if abs(x) <= 1 and abs(y) <= 1),
        "hcsp": sum(at(x, y) for x, y in ((0, 0), (-1, 0), (1, 0), (0, -1), (0, 1), (-2, 0), (2, 0))),
    }


def eq12_statistic(values):
    """The numbers printed as eq. (1)-(2): the mean and the sample standard
    deviation (n - 1) of the tabulated values A(d) themselves (the mean is
    therefore about 1 / (2R + 1)).  Table III reproduces them exactly, with the
    two deviations exchanged between f_x and f_y in the paper's print."""
    v = np.asarray(values, dtype=np.float64)
    return float(v.mean()), float(v.std(ddof=1))


def moments(values):
    """Mean and variance of the displacement d under the distribution A(d)."""
    v = np.asarray(values, dtype=np.float64)
    R = (v.size - 1) // 2
    d = np.arange(-R, R + 1)
    p = v / v.sum()
    mu = float((p * d).sum())
    return mu, float((p * (d - mu) ** 2).sum())


def d1(d1_counts, p):
    """Eq. (4): the distribution of the global best-matched point (FS MV) over
    the window, for the blocks whose current best-matched point in S1 is p."""
    c = np.asarray(d1_counts[S1.index(tuple(p))], dtype=np.float64)
    return c / max(c.sum(), 1.0)


def d2(d2_counts, R, qs):
    """Eq. (6): the distribution of the current best-matched point over the
    5x5 square S2 (returned as [dy + 2, dx + 2]), for the blocks whose global
    best-matched point is in the set qs (an (dx, dy) or a list of them)."""
    if isinstance(qs, tuple):
        qs = [qs]
    acc = np.zeros(25)
    for dx, dy in qs:
        if abs(dx) <= R and abs(dy) <= R:
            acc += d2_counts[dy + R, dx + R]
    return (acc / max(acc.sum(), 1.0)).reshape(5, 5)
