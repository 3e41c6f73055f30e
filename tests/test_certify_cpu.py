"""The full-size certification helper (tests/certify.py) on CPU: it accepts the oracle's own
converged result and rejects plausible wrong ones (a value moved at one state, a policy entry
changed where the margin is clear, a residual claimed smaller than it was, a sweep output off
by a little)."""
import numpy as np
import pytest

import mdp_synth
import oracle
from tests.certify import certify_solution, check_sweep


@pytest.fixture(scope="module")
def solved():
    syn = mdp_synth.ell_uniform(400, 5, 8, 0.99, seed=31)
    m = oracle.from_synth(syn)
    ref = oracle.gmres_policy_iteration(m, alpha=0.1, W=30, tol=1e-8)
    assert ref.status == "ok"
    return m, ref


def test_accepts_the_oracles_result(solved):
    m, ref = solved
    sw, bound = certify_solution(m, ref.v, ref.pi, ref.residual, 1e-6)
    assert bound <= 1e-6
    check_sweep(sw, sw.Tv, sw.pi, sw.res_inf)


def test_rejects_a_moved_value(solved):
    m, ref = solved
    v = ref.v.copy()
    v[123] += 1e-5
    with pytest.raises(AssertionError):
        certify_solution(m, v, ref.pi, ref.residual, 1e-6)


def test_rejects_a_changed_policy_entry(solved):
    m, ref = solved
    sw = oracle.bellman(m, ref.v)
    s = int(np.argmax(sw.margin))
    pi = ref.pi.copy()
    pi[s] = (pi[s] + 1) % m.A
    with pytest.raises(AssertionError):
        certify_solution(m, ref.v, pi, ref.residual, 1e-6)


def test_rejects_an_understated_residual(solved):
    m, ref = solved
    with pytest.raises(AssertionError):
        certify_solution(m, ref.v, ref.pi, ref.residual / 100.0, 1e-6)


def test_rejects_a_loose_value_tolerance(solved):
    m, ref = solved
    with pytest.raises(AssertionError):
        certify_solution(m, ref.v, ref.pi, ref.residual, 1e-12)


def test_sweep_check_rejects_small_errors(solved):
    m, ref = solved
    sw = oracle.bellman(m, ref.v)
    Tv = sw.Tv.copy()
    Tv[7] *= 1 + 1e-10
    with pytest.raises(AssertionError):
        check_sweep(sw, Tv, sw.pi, sw.res_inf)
    pi = sw.pi.copy()
    s = int(np.argmax(sw.margin))
    pi[s] = (pi[s] + 1) % m.A
    with pytest.raises(AssertionError):
        check_sweep(sw, sw.Tv, pi, sw.res_inf)
