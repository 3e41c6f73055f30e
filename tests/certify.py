"""Element-wise certification of a solve result by one oracle Bellman sweep (test helper).

A solver of this library returns v = T(V_K), pi = GreedyPolicy(V_K) and r = ||T V_K - V_K||_inf
(Alg. 2 with the outer stop of reading A1 and the output of reading A7).  One FP64 oracle sweep
at v then pins every state of the result, whatever S is:

  * residual: T is a gamma-contraction in the inf-norm (Sec. 2), so
    ||T v - v|| = ||T(T V_K) - T V_K|| <= gamma ||T V_K - V_K|| = gamma r.  The oracle's sweep at
    v must show that, up to rounding of the returned values (about 2^-48 relative in the
    double-float path, 2^-52 in FP64) and of the oracle's own FP64 sums.
  * value: for any V, ||V - V*||_inf <= ||T V - V||_inf / (1 - gamma) (contraction plus the
    inverse bound of Sec. 3.2, pinned on CPU by test_error_bound_from_residual), so the sweep
    bounds the error of v against the exact V* at EVERY state; it must be within the stated
    relative tolerance of max |v|.
  * policy: the returned pi is greedy at V_K, and each Q-value at V_K differs from the oracle's
    Q-value at v = T V_K by at most gamma ||V_K - T V_K|| = gamma r.  So pi must equal the
    oracle's greedy policy at v wherever the oracle's gap between the two best Q-values exceeds
    2 gamma r (and the 1e-9 relative rule for ties); everywhere the chosen action's Q-value
    must be within that gap of the best.

The same sweep, handed the library's own Bellman sweep at v, checks the sweep element by element
(Tv within 1e-12 relative, pi bit-exact where the margin exceeds 1e-9 relative).
"""
from __future__ import annotations

import numpy as np

import oracle


def vmax(v) -> float:
    return max(1.0, float(np.max(np.abs(v)))) if len(v) else 1.0


def certify_solution(m, v, pi, res_gpu: float, rtol_v: float, sw=None):
    """Assert the three properties above for the result (v, pi, r = res_gpu) of an MDP m.
    Returns the oracle sweep at v (reusable) and the certified bound on max|v - V*| / max|v|."""
    v = np.asarray(v, np.float64)
    pi = np.asarray(pi)
    sw = oracle.bellman(m, v) if sw is None else sw
    g = m.gamma
    vm = vmax(v)
    rounding = 1e-12 * vm
    assert sw.res_inf <= g * res_gpu + rounding, (sw.res_inf, g * res_gpu)
    bound = (sw.res_inf / (1.0 - g)) / vm
    assert bound <= rtol_v, bound
    Q = sw.Q
    cols = np.arange(m.S)
    q1 = Q[sw.pi, cols]
    thr = np.maximum(1e-9 * np.maximum(1.0, np.abs(q1)), 2.0 * g * res_gpu + rounding)
    sure = sw.margin > thr
    bad = int(np.sum(pi[sure] != sw.pi[sure]))
    assert bad == 0, f"{bad} of {int(sure.sum())} clear-margin policy entries differ"
    chosen = Q[pi, cols]
    assert np.all(chosen - q1 <= thr), float(np.max(chosen - q1 - thr))
    return sw, bound


def check_sweep(sw, Tv, pi, res, tol=1e-12):
    """The library's Bellman sweep (Tv, pi, ||Tv - v||) at the v of the oracle sweep sw:
    Tv within tol relative, the residual likewise, pi bit-exact where the oracle's margin
    exceeds 1e-9 * max(1, |Q1|) and within that margin elsewhere."""
    Tv = np.asarray(Tv, np.float64)
    pi = np.asarray(pi)
    scale = vmax(sw.Tv)
    assert float(np.max(np.abs(Tv - sw.Tv))) <= tol * scale
    assert abs(res - sw.res_inf) <= tol * scale
    Q = sw.Q
    cols = np.arange(Q.shape[1])
    q1 = Q[sw.pi, cols]
    thr = 1e-9 * np.maximum(1.0, np.abs(q1))
    sure = sw.margin > thr
    assert np.array_equal(pi[sure], sw.pi[sure])
    assert np.all(Q[pi, cols] - q1 <= thr + 1e-12)
