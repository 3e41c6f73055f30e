"""Plain, slow, FP64 CPU oracle for inexact GMRES policy iteration.

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's CPU-baseline leg
may import this package; the GPU library never imports, links or calls it, and shares no
code with it.  Every function cites the passage of the paper (Gargiani, Liao-McPherson,
Zanelli, Lygeros, "Inexact GMRES Policy Iteration for Large-Scale Markov Decision
Processes") that it writes out.

Pins (checked by the CPU tests against facts independent of this code): brute-force
enumeration of every policy on tiny MDPs in exact rational arithmetic, the truncated
series definition of the cost of a policy (Eq. "cost of pi"), closed forms for
single-state, absorbing and constant-cost MDPs, shift/scale/relabelling invariances of T
(Sec. 2), the spectrum, Lipschitz and inverse-norm lemmas (Sec. 3.1-3.2), GMRES's finite
termination in exact arithmetic (Sec. 2.2) and PI's finite termination (Sec. 2.1).
Parity unpinned: none of the functions exported here.
"""
from .mdp_oracle import (  # noqa: F401
    MDP, q_values, greedy_policy, bellman, policy_matrix, policy_cost, jacobian,
    policy_evaluation, brute_force, value_iteration, policy_iteration,
    optimistic_policy_iteration, gmres_policy_iteration, policy_eval_gmres, inner_threshold,
    inexact_pi_vi, two_level,
    bellman_residual, from_synth,
)
