"""Exact-rational restatement of the Voronoi merge (Sec. 3, Steps 1-7).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Every input float is converted to a ``fractions.Fraction`` (exactly), and every
decision is taken in exact arithmetic, so the partition this module returns is
the unique one that the paper's steps define for the given inputs.  Square
roots are avoided by comparing squares of non-negative quantities:

* Step 3, position axis:  sigma/L <= T   <=>  var <= T^2 L^2
* Step 3, momentum axis:  sigma/|P| <= T <=>  var <= T^2 P^2  (P != 0)
* Step 4: argmax of Delta^2 (position var/L^2, momentum var/P^2, +inf when
  P == 0 < var), lowest axis on exact ties.
* Step 5: q <= Q exactly.

Variants (the bits of ``variant``, as in the C oracle): ``VAR_NORMALIZED``
maximises (Delta_l / T_l)^2 = Delta_l^2 / T_l^2 in Step 4 (+inf for T_l = 0
< Delta_l, 0 for Delta_l = 0); ``VAR_PNORM`` takes the momentum scale |P|^2 =
sum of P_l^2 over the momentum axes in place of P_l^2.

Pure-Python loops: meant for cells of at most a few dozen particles.
"""
from __future__ import annotations

from fractions import Fraction

INF = float("inf")
VAR_NORMALIZED = 2
VAR_PNORM = 4


def _frac(x):
    return Fraction(float(x))


def _moments(q, w, members):
    W = sum(w[i] for i in members)
    Q = [sum(w[i] * ql[i] for i in members) / W for ql in q]
    var = [sum(w[i] * (ql[i] - Ql) ** 2 for i in members) / W for ql, Ql in zip(q, Q)]
    return W, Q, var


def _delta2(l, dx, var, scale2, L):
    """Delta_l squared (exact), +inf encoded as None; scale2 is the squared
    momentum scale (P_l^2, or |P|^2)."""
    if l < dx:
        return var / (L[l] * L[l])
    if var == 0:
        return Fraction(0)
    if scale2 == 0:
        return None
    return var / scale2


def _score(d2, T2):
    """(Delta / T)^2 for the normalised split axis; None is +inf."""
    if d2 is None:
        return None
    if d2 == 0:
        return Fraction(0)
    if T2 == 0:
        return None
    return d2 / T2


def _gt(a, b):
    """a > b for squared CVs where None stands for +inf."""
    if a is None:
        return b is not None
    if b is None:
        return False
    return a > b


def split_set(pos, mom, w, cell_size=(1.0, 1.0, 1.0), tol_x=0.1, tol_p=0.1, variant=0):
    """Leaves of one set, each a list of member ids in input order, in
    V1-first depth-first order, with their exact centroids (W, X+P)."""
    dx, dp = len(pos), len(mom)
    D = dx + dp
    q = [[_frac(v) for v in row] for row in list(pos) + list(mom)]
    wf = [_frac(v) for v in w]
    L = [_frac(v) for v in cell_size]
    T2 = [(_frac(tol_x) if l < dx else _frac(tol_p)) ** 2 for l in range(D)]
    leaves = []

    def rec(members):
        W, Q, var = _moments(q, wf, members)
        pn2 = sum(Q[l] * Q[l] for l in range(dx, D))
        d2 = [_delta2(l, dx, var[l], pn2 if variant & VAR_PNORM else Q[l] * Q[l], L)
              for l in range(D)]
        stop = all(d is not None and d <= T2[l] for l, d in enumerate(d2))
        if stop:
            if len(members) == 1:
                i = members[0]
                leaves.append((members, wf[i], [q[l][i] for l in range(D)]))
            else:
                leaves.append((members, W, Q))
            return
        key = [_score(d2[l], T2[l]) for l in range(D)] if variant & VAR_NORMALIZED else d2
        k = 0
        for l in range(1, D):
            if _gt(key[l], key[k]):
                k = l
        v1 = [i for i in members if q[k][i] <= Q[k]]
        v2 = [i for i in members if q[k][i] > Q[k]]
        assert v1 and v2, "exact cut cannot leave a side empty"
        rec(v1)
        rec(v2)

    rec(list(range(len(w))))
    return leaves


def merge(cell, pos, mom, w, n_cells, cell_size=(1.0, 1.0, 1.0), n_min=0,
          tol_x=0.1, tol_p=0.1, variant=0):
    """All cells: returns (index[n], centroids list of (cell, W, coords))
    with output slots in canonical order (cells ascending, leaves in
    V1-first depth-first order)."""
    n = len(cell)
    index = [None] * n
    out = []
    for c in range(int(n_cells)):
        members = [i for i in range(n) if int(cell[i]) == c]
        if not members:
            continue
        if len(members) <= n_min or len(members) == 1:
            for i in members:
                index[i] = len(out)
                out.append((c, _frac(w[i]),
                            [_frac(pos[l][i]) for l in range(len(pos))] +
                            [_frac(mom[l][i]) for l in range(len(mom))]))
            continue
        sub_pos = [[pos[l][i] for i in members] for l in range(len(pos))]
        sub_mom = [[mom[l][i] for i in members] for l in range(len(mom))]
        sub_w = [w[i] for i in members]
        for local, W, coords in split_set(sub_pos, sub_mom, sub_w, cell_size, tol_x, tol_p,
                                          variant):
            for j in local:
                index[members[j]] = len(out)
            out.append((c, W, coords))
    return index, out
