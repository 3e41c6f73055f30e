"""Exact rational arithmetic for tiny MDPs: an independent check on the FP64 oracle.

V^pi is the unique solution of (I - gamma P^pi) V = g^pi (Sec. 2.1); here it is solved by
Gauss-Jordan elimination over Python Fractions, so there is no rounding at all, and V* is
the elementwise minimum over every policy (Eq. optimal cost).
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np


def _solve(M, b):
    n = len(b)
    aug = [list(M[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if aug[r][c] != 0)
        aug[c], aug[p] = aug[p], aug[c]
        piv = aug[c][c]
        aug[c] = [x / piv for x in aug[c]]
        for r in range(n):
            if r != c and aug[r][c] != 0:
                f = aug[r][c]
                aug[r] = [x - f * y for x, y in zip(aug[r], aug[c])]
    return [aug[i][n] for i in range(n)]


def policy_value(P, g, gamma, pi):
    """P[a][s][s'], g[a][s], gamma as Fractions; returns V^pi as a list of Fractions."""
    n = len(pi)
    M = [[(Fraction(1) if i == j else Fraction(0)) - gamma * P[pi[i]][i][j] for j in range(n)]
         for i in range(n)]
    return _solve(M, [g[pi[i]][i] for i in range(n)])


def optimal(P, g, gamma, allowed=None):
    """Exact V* and the set of optimal policies by enumeration."""
    A, n = len(P), len(P[0])
    choices = allowed if allowed is not None else [list(range(A))] * n
    best = None
    table = []
    for pi in itertools.product(*choices):
        v = policy_value(P, g, gamma, pi)
        table.append((pi, v))
        best = v if best is None else [min(x, y) for x, y in zip(best, v)]
    opt = [pi for pi, v in table if v == best]
    return best, opt


def rational_mdp(S, A, seed, denom=7, cost_denom=5):
    """Random MDP whose transition rows and costs are small-denominator rationals; returns
    (P_frac, g_frac, P_float, g_float)."""
    rng = np.random.default_rng(seed)
    Pf, gf = [], []
    for a in range(A):
        rows = []
        for s in range(S):
            w = rng.integers(0, denom, size=S)
            if w.sum() == 0:
                w[rng.integers(0, S)] = 1
            tot = int(w.sum())
            rows.append([Fraction(int(x), tot) for x in w])
        Pf.append(rows)
        gf.append([Fraction(int(x), cost_denom) for x in rng.integers(0, 3 * cost_denom, size=S)])
    Pd = np.array([[[float(x) for x in r] for r in rows] for rows in Pf])
    gd = np.array([[float(x) for x in r] for r in gf])
    return Pf, gf, Pd, gd
