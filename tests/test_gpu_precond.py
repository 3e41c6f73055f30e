"""Two-level preconditioned inner solves (mdp_opts.precond_block) on the GPU.

The oracle's preconditioned iGMRES-PI (right-preconditioned GMRES on J^pi M^{-1} with
M^{-1} q = q + Pr J_c^{-1} R q over blocks of b consecutive states, the extension named in
Sec. 5) fixes what the path computes.  A preconditioner changes the Krylov space, not the fixed
point, so values meet the tolerances of the plain solves (written here, derived as in the
other parity tests): FP64 within 1e-10 relative with tol tightened so that
gamma*tol/(1-gamma) stays below it, mixed within 1e-6 relative at ||T(v)-v||_inf <= 1e-8;
policies bit-exact where the oracle's margin is clear.
"""
import numpy as np
import pytest

import mdp_synth
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_04299_gb300 import build
    build.build()
    import paper_2211_04299_gb300 as mg
    return mg


def rel_err(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def check_policy(pi_gpu, sw):
    Q = sw.Q
    q1 = np.min(Q, axis=0)
    sure = sw.margin > 1e-9 * np.maximum(1.0, np.abs(q1))
    assert np.array_equal(np.asarray(pi_gpu)[sure], sw.pi[sure])
    chosen = Q[np.asarray(pi_gpu), np.arange(Q.shape[1])]
    assert np.all(chosen - q1 <= 1e-9 * np.maximum(1.0, np.abs(q1)) + 1e-12)


def banded(S, prec, seed=1003, halfwidth=512, shift=64):
    return mdp_synth.ell_banded(S, 16, 32, halfwidth, shift, 0.999, seed=seed,
                                val_dtype=np.float32 if prec == "mixed" else np.float64)


# S=6000: 23 full blocks of 256 and a ragged one of 112; blocks of 64 leave a ragged 48
# and a coarse half-bandwidth of 17 blocks.
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("block", [256, 64])
def test_precond_banded_matches_oracle(mg, prec, block):
    syn = banded(6000, prec)
    m = oracle.from_synth(syn)
    ref = oracle.policy_iteration(m, tol=1e-11)
    h = mg.from_synth(syn)
    tol = 1e-8 if prec == "mixed" else 1e-11
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=tol, precision=prec, precond_block=block))
    assert st["status"] == 0 and st["residual_inf"] <= tol, st
    assert rel_err(v, ref.v) <= (1e-6 if prec == "mixed" else 1e-10)
    check_policy(pi, oracle.bellman(m, ref.v))
    # the coarse correction cuts the Krylov work several-fold, as in the oracle
    _, _, st0 = mg.ipi_solve(h, mg.opts(tol=tol, precision=prec))
    assert st["inner"] * 2 <= st0["inner"], (st["inner"], st0["inner"])
    h.close()


def test_precond_step_counts_follow_the_oracle(mg):
    """FP64: the GPU's preconditioned solve stops where the oracle's does, up to the rounding
    of the estimate that stands in for the true residual."""
    syn = banded(6000, "fp64")
    m = oracle.from_synth(syn)
    ref = oracle.gmres_policy_iteration(m, alpha=0.1, W=30, tol=1e-11, precond_block=256)
    ref0 = oracle.gmres_policy_iteration(m, alpha=0.1, W=30, tol=1e-11)
    assert ref.inner * 2 <= ref0.inner
    h = mg.from_synth(syn)
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=1e-11, precision="fp64", precond_block=256))
    assert st["status"] == 0
    assert abs(st["outer"] - ref.outer) <= 2, (st["outer"], ref.outer)
    assert st["inner"] <= 1.5 * ref.inner + 5, (st["inner"], ref.inner)
    assert rel_err(v, ref.v) <= 1e-9
    h.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_precond_graph_host_loop_and_reruns_agree(mg, prec):
    """Every kernel of the preconditioner sums in a fixed order, so the graph-resident loop,
    the host-driven loop and a second run agree bit for bit."""
    syn = banded(3000, prec, seed=5, halfwidth=200, shift=40)
    h = mg.from_synth(syn)
    tol = 1e-9 if prec == "mixed" else 1e-11
    o = dict(tol=tol, precision=prec, precond_block=128)
    v1, pi1, st1 = mg.ipi_solve(h, mg.opts(**o))
    v2, pi2, st2 = mg.ipi_solve(h, mg.opts(flags=mg.MDP_FLAG_HOST_LOOP, **o))
    v3, pi3, st3 = mg.ipi_solve(h, mg.opts(**o))
    for v, pi, st in ((v2, pi2, st2), (v3, pi3, st3)):
        assert st["status"] == 0
        np.testing.assert_array_equal(v1, v)
        np.testing.assert_array_equal(pi1, pi)
        assert (st1["inner"], st1["outer"]) == (st["inner"], st["outer"])
    h.close()


def test_precond_single_block_and_tiny(mg):
    """One aggregate (b >= S): J_c is the scalar 1 - gamma (row sums of P^pi are 1), so the
    coarse correction adds the mean of q / (1 - gamma); and S below a vector unit."""
    for S, b in ((700, 1024), (3, 4)):
        syn = mdp_synth.tiny_random(S, 3, seed=S, gamma=0.99, kind="ell", k=min(S, 4),
                                    density=0.5, val_dtype=np.float64)
        m = oracle.from_synth(syn)
        ref = oracle.policy_iteration(m, tol=1e-12)
        h = mg.from_synth(syn)
        v, pi, st = mg.ipi_solve(h, mg.opts(tol=1e-12, precision="fp64", precond_block=b))
        assert st["status"] == 0
        assert rel_err(v, ref.v) <= 1e-9
        check_policy(pi, oracle.bellman(m, ref.v))
        h.close()


def test_precond_rejections(mg):
    dense = mdp_synth.tiny_random(50, 2, seed=1, gamma=0.9, kind="dense", val_dtype=np.float64)
    h = mg.from_synth(dense)
    with pytest.raises(mg.MDPError, match="ELL"):
        mg.ipi_solve(h, mg.opts(precision="fp64", precond_block=16))
    h.close()
    syn = banded(3000, "fp64", seed=5, halfwidth=200, shift=40)
    h = mg.from_synth(syn)
    for bad in (3, 2, 1 << 21, -4):
        with pytest.raises(mg.MDPError, match="precond_block"):
            mg.ipi_solve(h, mg.opts(precision="fp64", precond_block=bad))
    with pytest.raises(mg.MDPError, match="ipi_solve only"):
        mg.vi_solve(h, mg.opts(precision="fp64", precond_block=64))
    with pytest.raises(mg.MDPError, match="ipi_solve only"):
        mg.ipi_vi_solve(h, mg.opts(precision="fp64", precond_block=64))
    # blocks of 4 states: transitions reach 100+ blocks away
    with pytest.raises(mg.MDPError, match="31 aggregation blocks"):
        mg.ipi_solve(h, mg.opts(precision="fp64", precond_block=4))
    # the handle still solves afterwards
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=1e-10, precision="fp64", precond_block=128))
    assert st["status"] == 0
    h.close()
    big = mdp_synth.ell_banded(40000, 2, 4, 8, 2, 0.9, seed=3, val_dtype=np.float64)
    h = mg.from_synth(big)
    with pytest.raises(mg.MDPError, match="8192"):
        mg.ipi_solve(h, mg.opts(precision="fp64", precond_block=4))
    h.close()


@pytest.mark.parametrize("W", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_precond_with_restarts_matches_oracle(mg, W, prec):
    """Short restart cycles (W = 2, 3) make inner solves restart from the candidate
    V_k + M^{-1} Q y, whose coarse part the combine kernel forms in RESTART mode."""
    syn = banded(3000, prec, seed=5, halfwidth=200, shift=40)
    m = oracle.from_synth(syn)
    ref = oracle.policy_iteration(m, tol=1e-11)
    refp = oracle.gmres_policy_iteration(m, alpha=0.1, W=W, tol=1e-10, precond_block=128)
    assert refp.restarts > 0
    h = mg.from_synth(syn)
    tol = 1e-8 if prec == "mixed" else 1e-10
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=tol, precision=prec, restart=W, precond_block=128))
    assert st["status"] == 0 and st["restarts"] > 0, st
    assert rel_err(v, ref.v) <= (1e-6 if prec == "mixed" else 1e-8)
    check_policy(pi, oracle.bellman(m, ref.v))
    if prec == "fp64":
        assert abs(st["outer"] - refp.outer) <= 2
    h.close()


def test_precond_inner_cap_reaches_the_same_fixed_point(mg):
    """An inner step cap (FINISH mode forms the capped candidate with its coarse part) slows
    the outer loop but not its fixed point."""
    syn = banded(3000, "fp64", seed=5, halfwidth=200, shift=40)
    m = oracle.from_synth(syn)
    ref = oracle.policy_iteration(m, tol=1e-11)
    h = mg.from_synth(syn)
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=1e-10, precision="fp64", max_inner=2,
                                        max_outer=500, precond_block=128))
    assert st["status"] == 0, st
    assert rel_err(v, ref.v) <= 1e-8
    check_policy(pi, oracle.bellman(m, ref.v))
    h.close()


# The device's coarse factorization (band build, GTH-form LU in FP32, explicit FP32 inverse)
# against the oracle's Galerkin J_c inverted in FP64.  Blocks of 128 give a half-bandwidth of at
# most 8 blocks (the single-thread register LU); blocks of 32 a wider band (the one-warp LU).
# Bound: 5e-6 of the largest entry, the FP32 GTH form's accuracy in the CPU restatement
# (tests/test_coarse_factor_cpu.py), at gamma up to 0.9999 where a plain LU would lose it.
@pytest.mark.parametrize("gamma", [0.999, 0.9999])
@pytest.mark.parametrize("block,narrow", [(128, True), (32, False)])
@pytest.mark.parametrize("vdt", [np.float32, np.float64])
def test_device_coarse_inverse_matches_oracle(mg, gamma, block, narrow, vdt):
    syn = mdp_synth.ell_banded(3000, 8, 16, 200, 40, gamma, seed=21, val_dtype=vdt)
    m = oracle.from_synth(syn)
    pi = oracle.bellman(m, np.zeros(syn.S)).pi
    _, _, Jc, _ = oracle.two_level(m, pi, block)
    exact = np.linalg.inv(Jc)
    h = mg.from_synth(syn)
    inv, bw = mg.precond_coarse_inverse(h, pi, block)
    h.close()
    assert inv.shape == Jc.shape
    assert (bw <= 8) == narrow, bw
    rel = float(np.max(np.abs(inv.astype(np.float64) - exact)) / np.max(np.abs(exact)))
    assert rel <= 5e-6, rel
    assert float(np.min(inv)) >= -1e-6 * float(np.max(inv))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_coarse_factor_reuse_gives_the_rebuilt_result(mg, prec):
    """Reusing the coarse factors of an earlier policy (default: while at most 1 in 1000 states
    changed action) and rebuilding them for every policy (MDP_FLAG_PC_REBUILD) both meet the
    oracle's values; the preconditioner only changes the Krylov space."""
    syn = banded(6000, prec, seed=1013)
    m = oracle.from_synth(syn)
    ref = oracle.policy_iteration(m, tol=1e-11)
    h = mg.from_synth(syn)
    tol = 1e-8 if prec == "mixed" else 1e-11
    bound = 1e-6 if prec == "mixed" else 1e-10
    for flags in (0, mg.MDP_FLAG_PC_REBUILD):
        v, pi, st = mg.ipi_solve(h, mg.opts(tol=tol, precision=prec, precond_block=256,
                                            flags=flags))
        assert st["status"] == 0 and st["residual_inf"] <= tol, (flags, st)
        assert rel_err(v, ref.v) <= bound
        check_policy(pi, oracle.bellman(m, ref.v))
    h.close()
