"""Brute-force enumeration of every alignment path (test infrastructure only).

An elastic distance of the common form (Eq. Common) is the minimum, over all
monotone lattice paths from (0,0) to (L_S, L_T) with unit steps diagonal,
down or right, of the sum of the step costs along the path: a diagonal step
into (i,j) costs Canonical(i,j), a down step AlternateRow(i,j) and a right
step AlternateColumn(i,j).  Border cells (i,0) / (0,j) are entered only by
down / right steps along the border; for +inf borders they are forbidden and
for ERP they cost cost(s_i,g) / cost(g,t_j) (Eq. ERP borders).  A window w
forbids interior cells with |i-j| > w and border cells with index > w + 1
(Alg. 4/5 initialise computed borders up to index w + 1).

This file enumerates the paths explicitly (no memoisation, so no dynamic
programming): it is exponential and only meant for lengths up to about 7.
The step costs are restated here from the paper's equations, independently
of ``eap_oracle.c``.
"""
from __future__ import annotations

import math

INF = math.inf


def _cost(kind_cost: int, a: float, b: float) -> float:
    d = a - b
    return d * d if kind_cost == 0 else abs(d)


def _msm_split_merge(c: float, new: float, x: float, y: float) -> float:
    # Eq. MSMCost: c when the new point lies between its two neighbours.
    lo, hi = (x, y) if x <= y else (y, x)
    if lo <= new <= hi:
        return c
    return c + min(abs(new - x), abs(new - y))


class StepCosts:
    """Step costs of one distance for series s, t (1-indexed via s[i-1])."""

    def __init__(self, kind: str, s, t, cost: int, window=None, g=0.05, wmax=1.0,
                 gap=0.0, msm_c=0.5, nu=0.001, lam=1.0):
        self.kind = kind
        self.s = [float(v) for v in s]
        self.t = [float(v) for v in t]
        self.cost = cost
        self.w = window
        self.g, self.wmax, self.gap, self.c, self.nu, self.lam = g, wmax, gap, msm_c, nu, lam
        self.L = max(len(self.s), len(self.t))

    def si(self, i):   # s_i with s_0 = 0
        return self.s[i - 1] if i >= 1 else 0.0

    def tj(self, j):
        return self.t[j - 1] if j >= 1 else 0.0

    def allowed(self, i, j) -> bool:
        if self.w is None:
            return True
        if i == 0 or j == 0:
            return max(i, j) <= self.w + 1
        return abs(i - j) <= self.w

    def border_down(self, i):   # entering (i,0) from (i-1,0)
        if self.kind == "erp" and self.allowed(i, 0):
            return _cost(self.cost, self.si(i), self.gap)
        return INF

    def border_right(self, j):  # entering (0,j) from (0,j-1)
        if self.kind == "erp" and self.allowed(0, j):
            return _cost(self.cost, self.gap, self.tj(j))
        return INF

    def diag(self, i, j):
        k = self.kind
        if k in ("dtw", "cdtw"):
            return _cost(self.cost, self.si(i), self.tj(j))
        if k == "wdtw":
            wt = self.wmax / (1.0 + math.exp(-self.g * (abs(i - j) - self.L / 2.0)))
            return wt * _cost(self.cost, self.si(i), self.tj(j))
        if k == "erp":
            return _cost(self.cost, self.si(i), self.tj(j))
        if k == "msm":
            return abs(self.si(i) - self.tj(j))
        if k == "twe":
            return (_cost(self.cost, self.si(i), self.tj(j))
                    + _cost(self.cost, self.si(i - 1), self.tj(j - 1))
                    + self.nu * (abs(i - j) + abs((i - 1) - (j - 1))))
        raise ValueError(k)

    def down(self, i, j):
        k = self.kind
        if k in ("dtw", "cdtw", "wdtw"):
            return self.diag(i, j)
        if k == "erp":
            return _cost(self.cost, self.si(i), self.gap)
        if k == "msm":
            return _msm_split_merge(self.c, self.si(i), self.si(i - 1), self.tj(j))
        if k == "twe":
            return _cost(self.cost, self.si(i), self.si(i - 1)) + self.nu * 1.0 + self.lam
        raise ValueError(k)

    def right(self, i, j):
        k = self.kind
        if k in ("dtw", "cdtw", "wdtw"):
            return self.diag(i, j)
        if k == "erp":
            return _cost(self.cost, self.tj(j), self.gap)
        if k == "msm":
            return _msm_split_merge(self.c, self.tj(j), self.si(i), self.tj(j - 1))
        if k == "twe":
            return _cost(self.cost, self.tj(j), self.tj(j - 1)) + self.nu * 1.0 + self.lam
        raise ValueError(k)


def all_paths(ls: int, lt: int):
    """Yield every monotone path from (0,0) to (ls,lt) as a list of
    (step, i, j) with step in {'d','v','h'} (the cell entered is (i,j))."""
    path = []

    def rec(i, j):
        if i == ls and j == lt:
            yield list(path)
            return
        if i < ls and j < lt:
            path.append(("d", i + 1, j + 1)); yield from rec(i + 1, j + 1); path.pop()
        if i < ls:
            path.append(("v", i + 1, j)); yield from rec(i + 1, j); path.pop()
        if j < lt:
            path.append(("h", i, j + 1)); yield from rec(i, j + 1); path.pop()

    yield from rec(0, 0)


def path_cost(sc: StepCosts, path) -> float:
    total = 0.0
    for step, i, j in path:
        if not sc.allowed(i, j):
            return INF
        if j == 0:
            c = sc.border_down(i)
        elif i == 0:
            c = sc.border_right(j)
        elif step == "d":
            c = sc.diag(i, j)
        elif step == "v":
            c = sc.down(i, j)
        else:
            c = sc.right(i, j)
        if c == INF:
            return INF
        total = total + c
    return total


def brute_distance(kind: str, s, t, cost: int, **kw) -> float:
    """Minimum path cost over all paths (exponential; lengths <= ~7)."""
    sc = StepCosts(kind, s, t, cost, **kw)
    best = INF
    for p in all_paths(len(sc.s), len(sc.t)):
        c = path_cost(sc, p)
        if c < best:
            best = c
    return best


def delannoy(m: int, n: int) -> int:
    """Number of such paths: the Delannoy number D(m,n)."""
    return sum(math.comb(m, k) * math.comb(n, k) * 2 ** k for k in range(min(m, n) + 1))
