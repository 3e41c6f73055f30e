"""Each test plants one plausible mistake in the CPU oracle (monkeypatched, on the CPU) and
checks that at least one pin in test_oracle_pins fails, so the pins are known to be able
to see that kind of error."""
import os

import numpy as np
import pytest

import oracle.mdp_oracle as mo
from tests import test_oracle_pins as pins


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_transposed_transition_is_caught(monkeypatch):
    def bad(mdp, a, v):
        if mdp.kind == "dense":
            return mdp.P[a].astype(np.float64).T @ v
        return mo.__dict__["_orig_ta"](mdp, a, v)
    monkeypatch.setitem(mo.__dict__, "_orig_ta", mo.transition_apply)
    monkeypatch.setattr(mo, "transition_apply", bad)
    _fails(pins.test_constant_cost_every_action_ties, "vi")


def test_dropped_discount_is_caught(monkeypatch):
    def bad(mdp, v):  # g + P v: the discount factor left out
        return np.stack([mdp.g[a] + mo.transition_apply(mdp, a, v) for a in range(mdp.A)])
    monkeypatch.setattr(mo, "q_values", bad)
    _fails(pins.test_single_state, "vi")


def test_argmax_instead_of_argmin_is_caught(monkeypatch):
    monkeypatch.setattr(mo, "greedy_policy", lambda Q: np.argmax(np.where(np.isfinite(Q), Q, -np.inf), axis=0).astype(np.int32))
    _fails(pins.test_golden_examples, os.path.join(pins.GOLDEN, "two_state_switch.json"), "pi")


def test_wrong_sign_in_gram_schmidt_is_caught(monkeypatch):
    orig_lsq = mo._lsq

    def bad_lsq(H, beta):
        y = orig_lsq(H, beta)
        return -y if H.shape[1] > 1 else y
    monkeypatch.setattr(mo, "_lsq", bad_lsq)
    _fails(pins.test_gmres_unrestarted_is_exact_within_n_steps, "dense")


def test_restart_that_drops_the_base_is_caught(monkeypatch):
    src = mo._gmres_inner

    def bad(J, g_pi, V_k, Phi_k, threshold, W, max_steps, st, minv=None):
        # restart from V_k every cycle (forgets the progress of earlier cycles)
        return src(J, g_pi, V_k, Phi_k, threshold, W, min(max_steps, W), st, minv)
    monkeypatch.setattr(mo, "_gmres_inner", bad)
    _fails(pins.test_gmres_restarted_converges_to_lu, 2)


def test_policy_matrix_with_wrong_row_index_is_caught(monkeypatch):
    orig = mo.policy_matrix

    def bad(mdp, pi):
        return orig(mdp, np.roll(np.asarray(pi), 1))
    monkeypatch.setattr(mo, "policy_matrix", bad)
    _fails(pins.test_golden_examples, os.path.join(pins.GOLDEN, "three_state_reset.json"), "igmres")


def test_forcing_sequence_that_ignores_the_residual_is_caught(monkeypatch):
    # alpha_k held at alpha whatever forcing_c says: convergence stays linear
    monkeypatch.setattr(mo, "inner_threshold", lambda alpha, c, phi, tol: alpha * phi)
    _fails(pins.test_adaptive_forcing_is_superlinear)


def test_forcing_sequence_with_max_instead_of_min_is_caught(monkeypatch):
    monkeypatch.setattr(mo, "inner_threshold",
                        lambda alpha, c, phi, tol: max(max(alpha, c * phi) * phi, 0.1 * tol)
                        if c > 0 else alpha * phi)
    _fails(pins.test_adaptive_forcing_is_superlinear)


def test_policy_rows_of_the_wrong_action_are_caught(monkeypatch):
    # every other P^pi built for an evaluation uses the next action's rows
    orig = mo.policy_matrix

    def drifting(mdp, pi):
        drifting.calls += 1
        return orig(mdp, pi) if drifting.calls % 2 else orig(mdp, (pi + 1) % mdp.A)
    drifting.calls = 0
    monkeypatch.setattr(mo, "policy_matrix", drifting)
    _fails(pins.test_inexact_pi_with_vi_inner_reduces_to_pi_and_vi, 0.9)


def _planted_two_level(kind):
    import scipy.linalg as sla
    import scipy.sparse as sp

    def bad(mdp, pi, block):
        J = mo.jacobian(mdp, pi)
        S = mdp.S
        agg = np.arange(S) // block
        if kind == "shift":
            agg = np.minimum(agg + (np.arange(S) % block == 0), agg[-1])
        nc = int(agg[-1]) + 1
        Pr = sp.csr_matrix((np.ones(S), (np.arange(S), agg)), shape=(S, nc))
        sizes = np.bincount(agg, minlength=nc).astype(np.float64)
        R = Pr.T.tocsr() if kind == "sum" else sp.diags(1.0 / sizes) @ Pr.T.tocsr()
        JPr = J @ Pr
        Jc = np.asarray((R @ JPr).todense() if sp.issparse(JPr) else R @ JPr)
        lu = sla.lu_factor(Jc)
        if kind == "no_identity":
            return R, Pr, Jc, lambda q: Pr @ sla.lu_solve(lu, R @ q)
        return R, Pr, Jc, lambda q: q + Pr @ sla.lu_solve(lu, R @ q)
    return bad


def test_restriction_that_sums_instead_of_averaging_is_caught(monkeypatch):
    import oracle
    monkeypatch.setattr(mo, "two_level", _planted_two_level("sum"))
    monkeypatch.setattr(oracle, "two_level", mo.two_level)
    _fails(pins.test_two_level_coarse_operator_is_the_galerkin_product)


def test_prolongation_into_the_wrong_block_is_caught(monkeypatch):
    import oracle
    monkeypatch.setattr(mo, "two_level", _planted_two_level("shift"))
    monkeypatch.setattr(oracle, "two_level", mo.two_level)
    _fails(pins.test_two_level_coarse_operator_is_the_galerkin_product)


def test_preconditioner_without_the_identity_term_is_caught(monkeypatch):
    import oracle
    monkeypatch.setattr(mo, "two_level", _planted_two_level("no_identity"))
    monkeypatch.setattr(oracle, "two_level", mo.two_level)
    _fails(pins.test_preconditioned_gmres_unrestarted_is_exact)
