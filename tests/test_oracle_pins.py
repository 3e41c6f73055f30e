"""Pins for the CPU oracle: facts fixed by the paper and by mathematics, independent of the
oracle's own code (exact rational brute force, the series definition of V^pi, closed
forms, invariances, the lemmas of Sec. 3 and finite termination)."""
import glob
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import MDP
import mdp_synth
from tests import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SOLVERS = {
    "vi": lambda m, tol: oracle.value_iteration(m, tol=tol),
    "pi": lambda m, tol: oracle.policy_iteration(m, tol=tol),
    "opi": lambda m, tol: oracle.optimistic_policy_iteration(m, W=5, tol=tol),
    "igmres": lambda m, tol: oracle.gmres_policy_iteration(m, alpha=0.1, W=3, tol=tol),
}


def dense_mdp(P, g, gamma, mask=None):
    P = np.asarray(P, np.float64)
    return MDP(S=P.shape[1], A=P.shape[0], gamma=float(gamma), g=np.asarray(g, np.float64),
               kind="dense", P=P, mask=mask)


def as_ell(m: MDP) -> MDP:
    """The same MDP in ELL storage with k = S (every column listed, in a shuffled order)."""
    rng = np.random.default_rng(0)
    col = np.empty((m.A, m.S, m.S), np.int32)
    val = np.empty((m.A, m.S, m.S))
    for a in range(m.A):
        for s in range(m.S):
            perm = rng.permutation(m.S)
            col[a, s] = perm
            val[a, s] = m.P[a, s, perm]
    return MDP(S=m.S, A=m.A, gamma=m.gamma, g=m.g, kind="ell", col=col, val=val, mask=m.mask)


# ------------------------------------------------------------------ golden, hand-derived

@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.json"))))
@pytest.mark.parametrize("solver", sorted(SOLVERS))
def test_golden_examples(path, solver):
    d = json.load(open(path))
    if d["kind"] == "dense":
        m = dense_mdp(d["P"], d["g"], d["gamma"])
    else:
        col = np.asarray(d["col"], np.int32)
        m = MDP(S=col.shape[1], A=col.shape[0], gamma=d["gamma"], g=np.asarray(d["g"], float),
                kind="ell", col=col, val=np.asarray(d["val"], float))
    r = SOLVERS[solver](m, 1e-13)
    assert r.status == "ok"
    np.testing.assert_allclose(r.v, d["v_star"], rtol=0, atol=1e-11)
    np.testing.assert_array_equal(r.pi, d["pi_star"])


# ------------------------------------------------------------------ exact brute force

@pytest.mark.parametrize("seed", range(12))
def test_brute_force_matches_exact_rational(seed):
    rng = np.random.default_rng(100 + seed)
    S, A = int(rng.integers(1, 5)), int(rng.integers(1, 4))
    gamma = Fraction(int(rng.integers(1, 10)), 10)
    Pf, gf, Pd, gd = exact.rational_mdp(S, A, seed)
    vstar_exact, opt = exact.optimal(Pf, gf, gamma)
    m = dense_mdp(Pd, gd, float(gamma))
    vstar, _ = oracle.brute_force(m)
    np.testing.assert_allclose(vstar, [float(x) for x in vstar_exact], rtol=1e-13, atol=1e-13)
    for name, solve in SOLVERS.items():
        r = solve(m, 1e-13)
        np.testing.assert_allclose(r.v, [float(x) for x in vstar_exact], rtol=1e-10, atol=1e-10,
                                   err_msg=name)
        # the returned policy must be one of the exactly optimal ones
        assert tuple(int(x) for x in r.pi) in {tuple(p) for p in opt}, name


@pytest.mark.parametrize("seed", range(4))
def test_brute_force_with_mask(seed):
    rng = np.random.default_rng(200 + seed)
    S, A = 3, 3
    Pf, gf, Pd, gd = exact.rational_mdp(S, A, 50 + seed)
    mask = rng.random((S, A)) < 0.6
    for s in range(S):
        mask[s, rng.integers(0, A)] = True
    allowed = [list(np.nonzero(mask[s])[0]) for s in range(S)]
    gamma = Fraction(4, 5)
    vstar_exact, opt = exact.optimal(Pf, gf, gamma, allowed)
    m = dense_mdp(Pd, gd, 0.8, mask=mask)
    for name, solve in SOLVERS.items():
        r = solve(m, 1e-13)
        np.testing.assert_allclose(r.v, [float(x) for x in vstar_exact], atol=1e-10, err_msg=name)
        assert all(mask[s, r.pi[s]] for s in range(S)), name
        assert tuple(int(x) for x in r.pi) in {tuple(p) for p in opt}, name


# ------------------------------------------------------------------ definitions

@pytest.mark.parametrize("kind", ["dense", "ell"])
def test_policy_evaluation_equals_series_definition(kind):
    """Eq. (cost of pi): V^pi = sum_t gamma^t (P^pi)^t g^pi, truncated once gamma^t < 1e-16."""
    syn = mdp_synth.tiny_random(12, 3, seed=7, gamma=0.7, kind=kind, k=4)
    m = oracle.from_synth(syn)
    pi = np.random.default_rng(1).integers(0, 3, size=12)
    Ppi = oracle.policy_matrix(m, pi)
    Ppi = Ppi.toarray() if sp.issparse(Ppi) else Ppi
    gpi = oracle.policy_cost(m, pi)
    acc, term = np.zeros(12), gpi.copy()
    for _ in range(200):
        acc += term
        term = 0.7 * (Ppi @ term)
    np.testing.assert_allclose(oracle.policy_evaluation(m, pi), acc, rtol=1e-13, atol=1e-13)


def test_q_values_by_hand_loops():
    """Q(s,a) = g(s,a) + gamma sum_s' p_ss'(a) V(s') with scalar loops over the ELL entries."""
    syn = mdp_synth.tiny_random(9, 4, seed=3, gamma=0.6, kind="ell", k=3)
    m = oracle.from_synth(syn)
    v = np.random.default_rng(2).normal(size=9)
    Q = oracle.q_values(m, v)
    for a in range(4):
        for s in range(9):
            ref = m.g[a, s]
            acc = 0.0
            for j in range(3):
                acc += m.val[a, s, j] * v[m.col[a, s, j]]
            assert abs(Q[a, s] - (ref + 0.6 * acc)) < 1e-14


def test_dense_and_ell_agree():
    syn = mdp_synth.tiny_random(6, 3, seed=11, gamma=0.9, kind="dense", density=0.5)
    m = oracle.from_synth(syn)
    e = as_ell(m)
    v = np.random.default_rng(5).normal(size=6)
    np.testing.assert_allclose(oracle.q_values(m, v), oracle.q_values(e, v), rtol=1e-14, atol=1e-14)
    r1 = oracle.gmres_policy_iteration(m, tol=1e-12)
    r2 = oracle.gmres_policy_iteration(e, tol=1e-12)
    np.testing.assert_allclose(r1.v, r2.v, rtol=1e-10)


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("solver", sorted(SOLVERS))
def test_single_state(solver):
    g = np.array([[0.7], [0.3], [0.9]])
    m = dense_mdp(np.ones((3, 1, 1)), g, 0.95)
    r = SOLVERS[solver](m, 1e-12)
    assert abs(r.v[0] - 0.3 / 0.05) < 1e-9 and r.pi[0] == 1


@pytest.mark.parametrize("solver", sorted(SOLVERS))
def test_absorbing_states(solver):
    rng = np.random.default_rng(9)
    S, A = 7, 4
    g = rng.random((A, S))
    P = np.broadcast_to(np.eye(S), (A, S, S)).copy()
    m = dense_mdp(P, g, 0.9)
    r = SOLVERS[solver](m, 1e-12)
    np.testing.assert_allclose(r.v, g.min(axis=0) / 0.1, rtol=1e-10)
    np.testing.assert_array_equal(r.pi, g.argmin(axis=0))


@pytest.mark.parametrize("solver", sorted(SOLVERS))
def test_constant_cost_every_action_ties(solver):
    """g = c gives V* = c/(1-gamma) for any row-stochastic P (the rows, not the columns,
    sum to one: a transposed P fails here) and every action ties up to rounding."""
    syn = mdp_synth.tiny_random(10, 3, seed=4, gamma=0.9, kind="dense", density=0.4)
    m = oracle.from_synth(syn)
    m.g = np.full((3, 10), 0.25)
    r = SOLVERS[solver](m, 1e-12)
    np.testing.assert_allclose(r.v, 2.5, rtol=1e-10)
    assert np.all(oracle.bellman(m, r.v).margin < 1e-12)


def test_exact_ties_take_the_lowest_index():
    """Reading of GreedyPolicy's tie-break: with P_a = I and equal costs the Q values tie
    exactly, and the lowest action index wins."""
    g = np.array([[1.0, 2.0, 0.5], [1.0, 1.0, 0.5], [3.0, 1.0, 0.5]])
    m = dense_mdp(np.broadcast_to(np.eye(3), (3, 3, 3)).copy(), g, 0.5)
    b = oracle.bellman(m, np.array([2.0, 2.0, 1.0]))
    np.testing.assert_array_equal(b.pi, [0, 1, 0])


# ------------------------------------------------------------------ invariances of T

def _solve_ref(m):
    return oracle.policy_iteration(m, tol=1e-13)


def test_shift_invariance():
    """T(V + c1) = TV + gamma c1 (Sec. 2): g + c gives V* + c/(1-gamma), same policy."""
    m = oracle.from_synth(mdp_synth.tiny_random(8, 3, seed=21, gamma=0.8))
    r0 = _solve_ref(m)
    m.g = m.g + 1.5
    r1 = _solve_ref(m)
    np.testing.assert_allclose(r1.v, r0.v + 1.5 / 0.2, rtol=1e-11)
    np.testing.assert_array_equal(r0.pi, r1.pi)


def test_scale_invariance():
    m = oracle.from_synth(mdp_synth.tiny_random(8, 3, seed=22, gamma=0.8))
    r0 = _solve_ref(m)
    m.g = 3.0 * m.g
    r1 = _solve_ref(m)
    np.testing.assert_allclose(r1.v, 3.0 * r0.v, rtol=1e-11)
    np.testing.assert_array_equal(r0.pi, r1.pi)


def test_relabelling_states():
    syn = mdp_synth.tiny_random(9, 3, seed=23, gamma=0.85)
    m = oracle.from_synth(syn)
    perm = np.random.default_rng(0).permutation(9)
    inv = np.argsort(perm)
    mp = dense_mdp(m.P[:, perm][:, :, perm], m.g[:, perm], m.gamma)
    r0, r1 = _solve_ref(m), _solve_ref(mp)
    np.testing.assert_allclose(r1.v, r0.v[perm], rtol=1e-11)
    np.testing.assert_array_equal(r1.pi, r0.pi[perm])
    assert np.array_equal(r1.v[inv], r0.v) or np.allclose(r1.v[inv], r0.v, rtol=1e-11)


# ------------------------------------------------------------------ lemmas of Sec. 3

@pytest.mark.parametrize("gamma", [0.5, 0.9, 0.99])
def test_spectrum_in_disc(gamma):
    """Lemma (Sec. 3): eigenvalues of I - gamma P^pi lie in the disc |z - 1| <= gamma."""
    syn = mdp_synth.tiny_random(30, 3, seed=31, gamma=gamma, density=0.3)
    m = oracle.from_synth(syn)
    for seed in range(3):
        pi = np.random.default_rng(seed).integers(0, 3, size=30)
        ev = np.linalg.eigvals(oracle.jacobian(m, pi))
        assert np.all(np.abs(ev - 1.0) <= gamma + 1e-12)


def test_residual_lipschitz():
    """Lemma (Sec. 3.2): ||r(V1) - r(V2)||_inf <= (1+gamma) ||V1 - V2||_inf."""
    m = oracle.from_synth(mdp_synth.tiny_random(15, 4, seed=41, gamma=0.9, kind="ell", k=5))
    rng = np.random.default_rng(3)
    for _ in range(50):
        v1, v2 = rng.normal(size=15) * 5, rng.normal(size=15) * 5
        lhs = np.max(np.abs(oracle.bellman_residual(m, v1) - oracle.bellman_residual(m, v2)))
        assert lhs <= 1.9 * np.max(np.abs(v1 - v2)) + 1e-12


def test_inverse_norm_bound():
    """Lemma (Sec. 3.2): ||(I - gamma P^pi)^{-1}||_inf <= 1/(1-gamma)."""
    m = oracle.from_synth(mdp_synth.tiny_random(20, 3, seed=43, gamma=0.95, density=0.2))
    for seed in range(5):
        pi = np.random.default_rng(seed).integers(0, 3, size=20)
        Jinv = np.linalg.inv(oracle.jacobian(m, pi))
        assert np.max(np.abs(Jinv).sum(axis=1)) <= 1 / 0.05 + 1e-9


def test_error_bound_from_residual():
    """gamma-contraction of T (Sec. 2): ||TV - V*||_inf <= gamma/(1-gamma) ||TV - V||_inf."""
    m = oracle.from_synth(mdp_synth.tiny_random(4, 3, seed=44, gamma=0.9))
    vstar, _ = oracle.brute_force(m)
    rng = np.random.default_rng(4)
    for _ in range(30):
        v = vstar + rng.normal(size=4)
        b = oracle.bellman(m, v)
        assert np.max(np.abs(b.Tv - vstar)) <= 0.9 / 0.1 * b.res_inf + 1e-12


# ------------------------------------------------------------------ GMRES (Sec. 2.2)

@pytest.mark.parametrize("kind", ["dense", "ell"])
def test_gmres_unrestarted_is_exact_within_n_steps(kind):
    """GMRES in exact arithmetic reaches the solution in at most n steps (Sec. 2.2)."""
    syn = mdp_synth.tiny_random(25, 3, seed=51, gamma=0.99, kind=kind, k=4)
    m = oracle.from_synth(syn)
    pi = np.random.default_rng(0).integers(0, 3, size=25)
    ref = oracle.policy_evaluation(m, pi)
    r = oracle.policy_eval_gmres(m, pi, target_inf=1e-12, W=40)
    assert r.inner <= 25 and r.restarts == 0
    np.testing.assert_allclose(r.v, ref, rtol=1e-10)


@pytest.mark.parametrize("W", [1, 2, 5])
def test_gmres_restarted_converges_to_lu(W):
    syn = mdp_synth.tiny_random(40, 2, seed=52, gamma=0.9, kind="ell", k=5)
    m = oracle.from_synth(syn)
    pi = np.random.default_rng(1).integers(0, 2, size=40)
    ref = oracle.policy_evaluation(m, pi)
    r = oracle.policy_eval_gmres(m, pi, v0=np.ones(40), target_inf=1e-12, W=W)
    assert r.status == "ok" and r.restarts >= 1
    np.testing.assert_allclose(r.v, ref, rtol=1e-10)


def test_gmres_one_step_on_absorbing_system():
    """With P^pi = I the system is (1 - gamma) V = g: the Krylov space of any residual is
    one-dimensional, so one step solves it (then H[2,1] = 0, a lucky breakdown)."""
    m = dense_mdp(np.broadcast_to(np.eye(5), (1, 5, 5)).copy(), np.arange(5.0)[None], 0.5)
    r = oracle.policy_eval_gmres(m, np.zeros(5, int), target_inf=1e-14, W=10)
    np.testing.assert_allclose(r.v, np.arange(5.0) / 0.5, rtol=1e-14)
    assert r.inner == 1


# ------------------------------------------------------------------ outer loops

def test_pi_finite_termination():
    """PI terminates in finitely many steps (Sec. 2.1), at most m^n policies."""
    for seed in range(6):
        m = oracle.from_synth(mdp_synth.tiny_random(4, 3, seed=60 + seed, gamma=0.95))
        r = oracle.policy_iteration(m, tol=0.0)
        assert r.status == "ok" and r.outer <= 3 ** 4
        vstar, _ = oracle.brute_force(m)
        np.testing.assert_allclose(r.v, vstar, rtol=1e-11)


def test_igmres_pi_stopping_rule_and_linear_rate():
    """Theorem (local contraction, Sec. 3.2): with alpha < (1-gamma)/(1+gamma), near V* the
    error contracts at least by (1+gamma)/(1-gamma) * alpha per outer step (up to a
    quadratic term); the residual history must fall at least that fast once close."""
    gamma = 0.8
    alpha = 0.5 * (1 - gamma) / (1 + gamma)
    m = oracle.from_synth(mdp_synth.tiny_random(60, 4, seed=71, gamma=gamma, kind="ell", k=6))
    vstar = oracle.policy_iteration(m, tol=1e-14).v
    errs = []
    # Alg. 1 with GMRES as the inner solver, one outer step at a time, recording
    # e_k = ||V_k - V*||_inf
    V = np.zeros(60)
    for k in range(8):
        b = oracle.bellman(m, V)
        errs.append(np.max(np.abs(V - vstar)))
        J = oracle.jacobian(m, b.pi)
        gpi = oracle.policy_cost(m, b.pi)
        Phi = gpi - J @ V
        if np.max(np.abs(Phi)) < 1e-12:
            break
        res = oracle.policy_eval_gmres(m, b.pi, v0=V,
                                       target_inf=alpha * np.max(np.abs(Phi)), W=30)
        assert np.max(np.abs(gpi - J @ res.v)) <= alpha * np.max(np.abs(Phi)) * (1 + 1e-12)
        V = res.v
    rate = (1 + gamma) / (1 - gamma) * alpha
    ratios = [errs[i + 1] / errs[i] for i in range(2, len(errs) - 1) if errs[i] > 1e-10]
    assert ratios and max(ratios) <= rate * 1.05


def test_adaptive_forcing_is_superlinear():
    """Theorem (local contraction, Sec. 3.2): a forcing sequence with alpha_k -> 0 gives
    Q-superlinear convergence, a constant alpha only Q-linear.  On the same MDP as the linear
    rate test: the constant-alpha residual ratios stay at the linear rate, the adaptive ones
    (alpha_k = min(alpha, ||Phi_k||_inf)) fall toward 0, and both reach V*."""
    gamma = 0.8
    alpha = 0.5 * (1 - gamma) / (1 + gamma)
    m = oracle.from_synth(mdp_synth.tiny_random(60, 4, seed=71, gamma=gamma, kind="ell", k=6))
    vstar = oracle.policy_iteration(m, tol=1e-14).v
    lin = oracle.gmres_policy_iteration(m, alpha=alpha, W=30, tol=1e-13)
    sup = oracle.gmres_policy_iteration(m, alpha=alpha, W=30, tol=1e-13, forcing_c=1.0)
    assert lin.status == "ok" and sup.status == "ok"
    r_lin = [lin.history[i + 1] / lin.history[i] for i in range(2, len(lin.history) - 1)]
    # ratios of steps that end well above the arithmetic's floor (the last step of a solve
    # to 1e-13 is limited by FP64 rounding, not by the forcing sequence)
    r_sup = [sup.history[i + 1] / sup.history[i] for i in range(2, len(sup.history) - 1)
             if sup.history[i + 1] >= 1e-12]
    rate = (1 + gamma) / (1 - gamma) * alpha
    assert max(r_lin) <= rate and min(r_lin) > 1e-2            # linear: bounded away from 0
    assert len(r_sup) >= 2 and all(b < a for a, b in zip(r_sup, r_sup[1:]))  # ratios shrink
    assert r_sup[-1] < 1e-3
    assert sup.outer < lin.outer
    for r in (lin, sup):
        np.testing.assert_allclose(r.v, vstar, rtol=0, atol=1e-11 * max(1.0, np.abs(vstar).max()))


def test_forcing_sequence_stays_in_range_and_vanishes():
    """alpha_k lies in [0, alpha] (the theorem's hypothesis) and alpha_k -> 0 as ||Phi_k||
    -> 0; the threshold never drops below tol / 10."""
    alpha, tol = 0.05, 1e-8
    for phi in (10.0, 1.0, 1e-2, 1e-4, 1e-6, 1e-9):
        thr = oracle.inner_threshold(alpha, 1.0, phi, tol)
        assert thr <= max(alpha * phi, 0.1 * tol) * (1 + 1e-15)
        assert thr >= 0.1 * tol
        assert oracle.inner_threshold(alpha, 0.0, phi, tol) == alpha * phi
    small = [oracle.inner_threshold(alpha, 1.0, phi, 0.0) / phi for phi in (1e-2, 1e-4, 1e-6)]
    assert small == sorted(small, reverse=True) and small[-1] <= 1e-6


@pytest.mark.parametrize("gamma", [0.9, 0.95])
def test_inexact_pi_with_vi_inner_reduces_to_pi_and_vi(gamma):
    """Alg. 1 with VI as the inner solver.  alpha -> 0: every evaluation is exact, so the outer
    iteration is PI's (same policies, same count).  alpha = (1+gamma)/2 > gamma: one
    application of T^{pi_k} already contracts the residual by gamma (T^{pi_k} V_k = T V_k), so
    each outer step takes exactly one inner step and the iterates are VI's, bit for bit."""
    m = oracle.from_synth(mdp_synth.tiny_random(80, 4, seed=3, gamma=gamma, kind="ell", k=6))
    pi_r = oracle.policy_iteration(m, tol=1e-12)
    exact = oracle.inexact_pi_vi(m, alpha=1e-14, tol=1e-12)
    assert exact.status == "ok" and exact.outer == pi_r.outer
    assert np.array_equal(exact.pi, pi_r.pi)
    np.testing.assert_allclose(exact.v, pi_r.v, rtol=0, atol=1e-10)
    vi_r = oracle.value_iteration(m, tol=1e-10)
    one = oracle.inexact_pi_vi(m, alpha=(1 + gamma) / 2, tol=1e-10, K=10000)
    assert one.inner == one.outer == vi_r.outer
    assert one.history == vi_r.history and np.array_equal(one.v, vi_r.v)
    mid = oracle.inexact_pi_vi(m, alpha=0.1, tol=1e-10)
    assert mid.status == "ok" and vi_r.outer > mid.outer > pi_r.outer
    assert np.max(np.abs(mid.v - pi_r.v)) <= gamma * 1e-10 / (1 - gamma) * 1.01


def test_two_level_coarse_operator_is_the_galerkin_product():
    """J_c[I][J] = (1/|I|) sum_{s in I} sum_{s' in J} J[s][s'] for consecutive blocks (the last
    one shorter), R Pr = I, and J_c = I - gamma P_c with P_c >= 0 row-stochastic."""
    syn = mdp_synth.tiny_random(37, 3, seed=12, gamma=0.9)
    m = oracle.from_synth(syn)
    pi = oracle.bellman(m, np.zeros(37)).pi
    R, Pr, Jc, _ = oracle.two_level(m, pi, 8)
    J = np.asarray(oracle.jacobian(m, pi))
    blocks = [list(range(i, min(i + 8, 37))) for i in range(0, 37, 8)]
    ref = np.array([[sum(J[s, t] for s in bi for t in bj) / len(bi) for bj in blocks]
                    for bi in blocks])
    np.testing.assert_allclose(Jc, ref, rtol=0, atol=1e-14)
    np.testing.assert_allclose((R @ Pr).toarray(), np.eye(len(blocks)), rtol=0, atol=1e-15)
    Pc = (np.eye(len(blocks)) - Jc) / 0.9
    assert np.all(Pc >= -1e-15)
    np.testing.assert_allclose(Pc.sum(axis=1), 1.0, rtol=0, atol=1e-13)


def test_preconditioned_gmres_unrestarted_is_exact():
    """Right-preconditioned GMRES without restarts (W >= n) solves J V = g^pi exactly within n
    steps, like plain GMRES (the preconditioner is nonsingular)."""
    syn = mdp_synth.tiny_random(30, 3, seed=13, gamma=0.95, kind="ell", k=5)
    m = oracle.from_synth(syn)
    pi = oracle.bellman(m, np.zeros(30)).pi
    exact = oracle.policy_evaluation(m, pi)
    r = oracle.policy_eval_gmres(m, pi, target_inf=1e-12, W=40, precond_block=4)
    assert r.status == "ok" and r.inner <= 30
    np.testing.assert_allclose(r.v, exact, rtol=0, atol=1e-10 * np.abs(exact).max())


def test_two_level_preconditioner_cuts_inner_steps():
    """Banded transitions with gamma = 0.999 (the growth-model shape): the slow modes of
    I - gamma P^pi are smooth over the state index, which the coarse correction removes; the
    preconditioned evaluation needs a tenth of the plain GMRES(30) steps or fewer."""
    syn = mdp_synth.ell_banded(20000, 4, 16, 512, 64, 0.999, seed=7, val_dtype=np.float32)
    m = oracle.from_synth(syn)
    pi = oracle.bellman(m, np.zeros(20000)).pi
    plain = oracle.policy_eval_gmres(m, pi, target_inf=1e-6, W=30)
    pre = oracle.policy_eval_gmres(m, pi, target_inf=1e-6, W=30, precond_block=128)
    assert plain.status == "ok" and pre.status == "ok"
    assert pre.inner * 10 <= plain.inner


def test_preconditioned_igmres_pi_matches_pi():
    syn = mdp_synth.ell_banded(3000, 16, 32, 512, 64, 0.999, seed=1003, val_dtype=np.float32)
    m = oracle.from_synth(syn)
    ref = oracle.policy_iteration(m, tol=1e-12)
    r = oracle.gmres_policy_iteration(m, alpha=0.1, W=30, tol=1e-10, precond_block=64)
    assert r.status == "ok"
    np.testing.assert_allclose(r.v, ref.v, rtol=0, atol=1e-10 * np.abs(ref.v).max() / (1 - 0.999))


@pytest.mark.parametrize("gamma", [0.9, 0.99])
def test_igmres_pi_agrees_with_pi_on_config_shaped_input(gamma):
    syn = mdp_synth.ell_uniform(300, 4, 8, gamma, seed=5)
    m = oracle.from_synth(syn)
    ref = oracle.policy_iteration(m, tol=1e-12)
    r = oracle.gmres_policy_iteration(m, alpha=0.1, W=30, tol=1e-12)
    assert r.status == "ok"
    np.testing.assert_allclose(r.v, ref.v, rtol=1e-10)
    sure = ref.margin > 1e-9 * np.maximum(1, np.abs(ref.v))
    np.testing.assert_array_equal(r.pi[sure], ref.pi[sure])


def test_paper_qualitative_ordering():
    """Sec. 4: PI needs the fewest outer iterations, then iGMRES-PI, then OPI; OPI improves
    with more inner steps W."""
    m = oracle.from_synth(mdp_synth.ell_uniform(400, 5, 8, 0.95, seed=8))
    pi = oracle.policy_iteration(m, tol=1e-8)
    ig = oracle.gmres_policy_iteration(m, alpha=0.1, W=30, tol=1e-8)
    o5 = oracle.optimistic_policy_iteration(m, W=5, tol=1e-8)
    o20 = oracle.optimistic_policy_iteration(m, W=20, tol=1e-8)
    assert pi.outer <= ig.outer <= o20.outer <= o5.outer


def test_gmres_steps_robust_to_gamma_vi_sweeps_not():
    """Fig. 2 (Sec. 3.1): policy evaluation at n = 100 by GMRES needs about the same number
    of Arnoldi steps from gamma = 0.5 to 0.999 (spectrum lemma: the eigenvalues of
    I - gamma P^pi lie in the disc of radius gamma around 1, and for a well-mixed P^pi all but
    one cluster near 1), while VI needs log(tol)/log(gamma) sweeps up to a constant: the
    Perron component of the residual shrinks by exactly gamma per sweep."""
    steps, sweeps = [], []
    for g in (0.5, 0.9, 0.99, 0.999):
        syn = mdp_synth.dense_dirichlet(100, 1, 1.0, g, seed=2022, dtype=np.float64)
        m = oracle.from_synth(syn)
        pi0 = np.zeros(100, np.int32)
        rg = oracle.policy_eval_gmres(m, pi0, target_inf=1e-8, W=64)
        rv = oracle.value_iteration(m, tol=1e-8, max_iter=10 ** 6)
        steps.append(rg.inner)
        sweeps.append(rv.outer)
        # VI: ||Phi_k||_inf >= gamma^k * |Perron component| with ||Phi_0|| = ||g|| <= 1
        assert rv.outer >= np.log(1e-8) / np.log(g) - np.log(1e3) / -np.log(g) - 1
        assert rv.outer <= np.log(1e-8) / np.log(g) + 5 / (1 - g)
    assert steps[-1] <= 2 * steps[0] + 2 and max(steps) <= 100
    assert sweeps[-1] >= 100 * sweeps[0]
