"""GPU-vs-oracle parity through the C ABI.

Tolerances (written here, derived from the arithmetic):
  * FP64 path: Bellman values within 1e-13 relative (a k-term FP64 dot product in a
    different order); solved values within 1e-10 relative with tol tightened so that the
    contraction bound gamma*tol/(1-gamma) stays below it.
  * mixed path: Bellman sweeps in double-float (about 2^-48 relative per operation) within
    1e-12 relative; solved values within 1e-6 relative at ||T(v)-v||_inf <= 1e-8.
  * policies: bit-exact wherever the oracle's gap between the two best Q-values exceeds
    1e-9 * max(1, |Q1|) (ties elsewhere may resolve either way in floating point); where
    the gap is smaller the GPU's action must still be within that gap of the best.
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


def check_policy(pi_gpu, sw, v=None):
    """pi bit-exact where the oracle margin is clear; elsewhere within the margin."""
    Q = sw.Q
    q1 = np.min(Q, axis=0)
    sure = sw.margin > 1e-9 * np.maximum(1.0, np.abs(q1))
    assert np.array_equal(np.asarray(pi_gpu)[sure], sw.pi[sure]), \
        f"{int(np.sum(np.asarray(pi_gpu)[sure] != sw.pi[sure]))} clear-margin mismatches"
    chosen = Q[np.asarray(pi_gpu), np.arange(Q.shape[1])]
    assert np.all(chosen - q1 <= 1e-9 * np.maximum(1.0, np.abs(q1)) + 1e-12)


def make(kind, S, A, k, seed, mask_frac=0.0, val_dtype=np.float64, gamma=0.9):
    return mdp_synth.tiny_random(S, A, seed, gamma=gamma, kind=kind, k=k, density=0.5,
                                 mask_frac=mask_frac, val_dtype=val_dtype)


# ------------------------------------------------------------------ Bellman sweep
CASES = [("ell", 1, 1, 1), ("ell", 3, 2, 2), ("ell", 33, 5, 7), ("ell", 257, 3, 16),
         ("ell", 1000, 4, 32), ("ell", 777, 16, 13), ("dense", 1, 3, None), ("dense", 3, 2, None),
         ("dense", 33, 5, None), ("dense", 130, 8, None), ("dense", 515, 9, None),
         ("dense", 1000, 3, None), ("dense", 70, 1, None), ("dense", 1031, 4, None),
         ("dense", 2049, 6, None), ("dense", 1500, 7, None)]


@pytest.mark.parametrize("kind,S,A,k", CASES)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("mask_frac", [0.0, 0.3])
def test_bellman_apply_parity(mg, kind, S, A, k, prec, mask_frac):
    vdt = np.float32 if prec == "mixed" else np.float64
    syn = make(kind, S, A, k, seed=S * 7 + A, mask_frac=mask_frac, val_dtype=vdt)
    m = oracle.from_synth(syn)
    h = mg.from_synth(syn)
    rng = np.random.default_rng(S)
    for trial in range(2):
        v = rng.normal(size=S) * (10.0 if trial else 1.0) + trial * 50
        sw = oracle.bellman(m, v)
        Tv, pi, res = mg.bellman_apply(h, v, precision=prec)
        tol = 1e-13 if prec == "fp64" else 1e-12
        assert rel_err(Tv, sw.Tv) <= tol
        assert abs(res - sw.res_inf) <= tol * max(1.0, np.max(np.abs(sw.Tv)))
        check_policy(pi, sw)
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bellman_device_pointers_and_margin(mg, prec):
    import torch
    vdt = np.float32 if prec == "mixed" else np.float64
    syn = make("ell", 300, 6, 5, seed=3, val_dtype=vdt)
    m = oracle.from_synth(syn)
    h = mg.from_synth(syn, device=True)
    v = np.random.default_rng(1).normal(size=300)
    sw = oracle.bellman(m, v)
    Tv, pi, res, margin = mg.bellman_apply(h, torch.from_numpy(v).cuda(), precision=prec,
                                           margin=True)
    assert rel_err(Tv.cpu().numpy(), sw.Tv) <= 1e-12
    mg_cpu = margin.cpu().numpy()
    fin = np.isfinite(sw.margin)
    assert np.allclose(mg_cpu[fin], sw.margin[fin], rtol=1e-9, atol=1e-11)
    check_policy(pi.cpu().numpy(), sw)


@pytest.mark.parametrize("S,A", [(16500, 2), (4100, 8)])
def test_bellman_dense_wide_rows(mg, S, A):
    """Rows longer than 16 pipeline stages (the accumulators fold into a double-word total)
    and a width just past a stage boundary, FP32 Dirichlet rows as at the bench size."""
    syn = mdp_synth.dense_dirichlet(S, A, 0.1, 0.99, seed=S + A)
    m = oracle.from_synth(syn)
    h = mg.from_synth(syn)
    v = np.random.default_rng(3).normal(size=S) * 30 + 50
    sw = oracle.bellman(m, v)
    Tv, pi, res = mg.bellman_apply(h, v, precision="mixed")
    assert rel_err(Tv, sw.Tv) <= 1e-12
    assert abs(res - sw.res_inf) <= 1e-12 * max(1.0, np.max(np.abs(sw.Tv)))
    check_policy(pi, sw)
    h.close()


def test_bellman_edge_cases(mg):
    # absorbing states: Tv = g_min + gamma v exactly representable
    S, A = 9, 3
    g = np.random.default_rng(0).random((A, S))
    P = np.broadcast_to(np.eye(S), (A, S, S)).copy()
    h = mg.mdp_create_dense(P, g, 0.5)
    v = np.arange(S, dtype=np.float64)
    for prec in ["fp64"]:
        Tv, pi, _ = mg.bellman_apply(h, v, precision=prec)
        np.testing.assert_allclose(Tv, g.min(0) + 0.5 * v, rtol=1e-15)
        np.testing.assert_array_equal(pi, g.argmin(0))
    # exact ties -> lowest index
    g2 = np.ones((A, S))
    h2 = mg.mdp_create_dense(P, g2, 0.5)
    Tv, pi, _ = mg.bellman_apply(h2, v, precision="fp64")
    np.testing.assert_array_equal(pi, 0)
    # k = S with every column listed
    syn = make("ell", 6, 2, 6, seed=9)
    h3 = mg.from_synth(syn)
    sw = oracle.bellman(oracle.from_synth(syn), np.ones(6))
    Tv, pi, _ = mg.bellman_apply(h3, np.ones(6), precision="fp64")
    assert rel_err(Tv, sw.Tv) <= 1e-13


def test_invalid_mdps_are_rejected(mg):
    S, A = 5, 2
    g = np.zeros((A, S))
    P = np.full((A, S, S), 1.0 / S)
    bad = P.copy(); bad[1, 2, 3] += 0.1
    with pytest.raises(mg.MDPError, match="sum"):
        mg.mdp_create_dense(bad, g, 0.9)
    bad = P.copy(); bad[0, 0, 0] = np.nan
    with pytest.raises(mg.MDPError):
        mg.mdp_create_dense(bad, g, 0.9)
    col = np.zeros((A, S, 1), np.int32); col[0, 0, 0] = S
    with pytest.raises(mg.MDPError, match="column"):
        mg.mdp_create_ell(col, np.ones((A, S, 1)), g, 0.9)
    mask = np.ones((S, A), np.uint8); mask[2] = 0
    with pytest.raises(mg.MDPError, match="allowed"):
        mg.mdp_create_dense(P, g, 0.9, mask)
    gn = g.copy(); gn[0, 1] = np.inf
    with pytest.raises(mg.MDPError, match="finite"):
        mg.mdp_create_dense(P, gn, 0.9)


# ------------------------------------------------------------------ policy evaluation
@pytest.mark.parametrize("kind", ["ell", "dense"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("W", [3, 30])
def test_policy_eval_gmres_parity(mg, kind, prec, W):
    vdt = np.float32 if prec == "mixed" else np.float64
    syn = make(kind, 400, 3, 9, seed=11, val_dtype=vdt, gamma=0.99)
    m = oracle.from_synth(syn)
    h = mg.from_synth(syn)
    pi = np.random.default_rng(2).integers(0, 3, size=400).astype(np.int32)
    ref = oracle.policy_evaluation(m, pi)
    target = 1e-9
    V, st = mg.policy_eval_gmres(h, pi, None, target, mg.opts(restart=W, precision=prec))
    assert st["status"] == 0, st
    Jv = oracle.policy_cost(m, pi) - oracle.jacobian(m, pi) @ V
    assert np.max(np.abs(Jv)) <= target * 1.0001
    # ||V - V^pi|| <= ||J^-1|| ||r|| <= target / (1 - gamma)
    assert np.max(np.abs(V - ref)) <= target / 0.01 * 1.01


# ------------------------------------------------------------------ solvers
SOLVER_NAMES = ["ipi_solve", "vi_solve", "pi_solve", "opi_solve", "ipi_vi_solve"]


@pytest.mark.parametrize("name", SOLVER_NAMES)
@pytest.mark.parametrize("kind", ["ell", "dense"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_small_solvers_match_brute_force_scale_oracle(mg, name, kind, prec):
    vdt = np.float32 if prec == "mixed" else np.float64
    syn = make(kind, 60, 4, 5, seed=21, val_dtype=vdt, gamma=0.9, mask_frac=0.2)
    m = oracle.from_synth(syn)
    ref = oracle.policy_iteration(m, tol=1e-13)
    h = mg.from_synth(syn)
    tol = 1e-12 if prec == "fp64" else 1e-10
    v, pi, st = getattr(mg, name)(h, mg.opts(tol=tol, precision=prec, opi_W=10,
                                              max_outer=5000))
    assert st["status"] == 0, st
    assert st["residual_inf"] <= tol
    assert rel_err(v, ref.v) <= (1e-10 if prec == "fp64" else 1e-9)
    check_policy(pi, oracle.bellman(m, ref.v))


def test_ipi_vi_limits_match_pi_and_vi(mg):
    """Inexact PI with VI inner steps (Alg. 1): alpha -> 0 evaluates exactly (PI's outer count
    and policy); alpha = (1+gamma)/2 takes one inner step per outer step (VI's count)."""
    syn = make("ell", 200, 4, 6, seed=8, gamma=0.9)
    m = oracle.from_synth(syn)
    h = mg.from_synth(syn)
    pi_r = oracle.policy_iteration(m, tol=1e-12)
    v, pi, st = mg.ipi_vi_solve(h, mg.opts(tol=1e-12, precision="fp64", alpha=1e-14,
                                           max_inner=5000))
    assert st["status"] == 0 and st["outer"] == pi_r.outer
    check_policy(pi, oracle.bellman(m, pi_r.v))
    _, _, st_vi = mg.vi_solve(h, mg.opts(tol=1e-10, precision="fp64", max_outer=5000))
    _, _, st1 = mg.ipi_vi_solve(h, mg.opts(tol=1e-10, precision="fp64", alpha=0.95,
                                           max_outer=5000))
    assert st1["status"] == 0 and st1["inner"] == st1["outer"] == st_vi["outer"]


def test_ipi_vi_config1_fp64_matches_oracle(mg):
    syn = mdp_synth.config(1)
    m = oracle.from_synth(syn)
    ref = oracle.inexact_pi_vi(m, alpha=0.1, tol=1e-13)
    h = mg.from_synth(syn)
    tol = 1e-10 * np.max(np.abs(ref.v)) * (1 - 0.95) / (2 * 0.95)
    v, pi, st = mg.ipi_vi_solve(h, mg.opts(tol=tol, precision="fp64", alpha=0.1))
    assert st["status"] == 0 and st["residual_inf"] <= tol
    assert rel_err(v, ref.v) <= 1e-10
    check_policy(pi, oracle.bellman(m, ref.v))


def test_ipi_config1_fp64_matches_oracle(mg):
    syn = mdp_synth.config(1)                      # S=2000, A=5, k=16, FP64, gamma=0.95
    m = oracle.from_synth(syn)
    ref = oracle.gmres_policy_iteration(m, alpha=0.1, W=30, tol=1e-13)
    h = mg.from_synth(syn)
    # tolerance tightened so that gamma*tol/(1-gamma) <= 1e-10 * ||v|| / 2
    tol = 1e-10 * np.max(np.abs(ref.v)) * (1 - 0.95) / (2 * 0.95)
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=tol, precision="fp64", alpha=0.1, restart=30))
    assert st["status"] == 0 and st["residual_inf"] <= tol
    assert rel_err(v, ref.v) <= 1e-10
    check_policy(pi, oracle.bellman(m, ref.v))
    # the outer loop is the paper's: a handful of outer iterations, inner work bounded
    assert st["outer"] <= ref.outer + 3


def test_ipi_config1_mixed_matches_oracle(mg):
    syn = mdp_synth.config(1)
    syn.val = syn.val.astype(np.float32)            # the FP32-stored MDP, read by both sides
    m = oracle.from_synth(syn)
    ref = oracle.gmres_policy_iteration(m, alpha=0.1, W=30, tol=1e-13)
    h = mg.from_synth(syn)
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=1e-8, precision="mixed"))
    assert st["status"] == 0 and st["residual_inf"] <= 1e-8
    assert rel_err(v, ref.v) <= 1e-6
    # certified: the oracle's T at the GPU's v is within gamma * 1e-8 of v
    assert oracle.bellman(m, v).res_inf <= 0.95e-8 * 1.01


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_ipi_dense_dirichlet_scaled(mg, prec):
    syn = mdp_synth.dense_dirichlet(1500, 8, 0.1, 0.99, seed=77,
                                    dtype=np.float32 if prec == "mixed" else np.float64)
    m = oracle.from_synth(syn)
    ref = oracle.policy_iteration(m, tol=1e-12)
    h = mg.from_synth(syn)
    tol = 1e-8 if prec == "mixed" else 1e-12
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=tol, precision=prec))
    assert st["status"] == 0
    assert rel_err(v, ref.v) <= (1e-6 if prec == "mixed" else 1e-10)
    check_policy(pi, oracle.bellman(m, ref.v))


@pytest.mark.parametrize("kind", ["ell", "dense"])
def test_ipi_graph_and_host_loop_agree(mg, kind):
    """The graph-resident inner loop and the host-driven one run the same kernels in the same
    order, so the solves agree bit for bit."""
    syn = make(kind, 700, 5, 9, seed=41, val_dtype=np.float32, gamma=0.99)
    h = mg.from_synth(syn)
    v1, pi1, st1 = mg.ipi_solve(h, mg.opts(tol=1e-9, precision="mixed"))
    v2, pi2, st2 = mg.ipi_solve(h, mg.opts(tol=1e-9, precision="mixed", flags=mg.MDP_FLAG_HOST_LOOP))
    assert st1["status"] == 0 and st2["status"] == 0
    np.testing.assert_array_equal(v1, v2)
    np.testing.assert_array_equal(pi1, pi2)
    assert st1["inner"] == st2["inner"] and st1["outer"] == st2["outer"]


def test_warm_start_is_resume(mg):
    syn = make("ell", 500, 4, 6, seed=5)
    h = mg.from_synth(syn)
    v1, _, st1 = mg.ipi_solve(h, mg.opts(tol=1e-4, precision="fp64"))
    v0 = np.ascontiguousarray(v1)
    v2, _, st2 = mg.ipi_solve(h, mg.opts(tol=1e-11, precision="fp64", v0=v0))
    v3, _, st3 = mg.ipi_solve(h, mg.opts(tol=1e-11, precision="fp64"))
    assert rel_err(v2, v3) <= 1e-10
    assert st2["outer"] <= st3["outer"]


@pytest.mark.parametrize("kind", ["ell", "dense"])
def test_async_loads_equal_sync_loads_and_report_invalid_data(mg, kind):
    """mdp_load_*_async enqueues the upload and validation; the next call on the handle waits
    for that handle's stream and reports the validation (invalid data -> EINVAL)."""
    import torch
    a = make(kind, 300, 4, 7, seed=51, val_dtype=np.float32, gamma=0.95)
    b = make(kind, 300, 4, 7, seed=52, val_dtype=np.float32, gamma=0.95)
    o = mg.opts(tol=1e-9, precision="mixed")

    def load(h, syn, asyn):
        pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()
        g = pin(syn.g)
        if kind == "dense":
            P = pin(syn.P)
            (mg.mdp_load_dense_async if asyn else mg.mdp_load_dense)(h, P, g)
            return (P, g)
        col, val = pin(syn.col), pin(syn.val)
        (mg.mdp_load_ell_async if asyn else mg.mdp_load_ell)(h, col, val, g)
        return (col, val, g)

    h0, h1 = mg.from_synth(a), mg.from_synth(a)
    keep = load(h0, b, False)
    v_ref, pi_ref, _ = mg.ipi_solve(h0, o)
    keep1 = load(h1, b, True)                  # enqueued ...
    keep2 = load(h0, a, True)                  # ... and another handle's load meanwhile
    v1, pi1, _ = mg.ipi_solve(h1, o)          # waits for h1's stream only
    np.testing.assert_array_equal(v1, v_ref)
    np.testing.assert_array_equal(pi1, pi_ref)
    v0, _, st0 = mg.ipi_solve(h0, o)
    va, _, _ = mg.ipi_solve(mg.from_synth(a), o)
    np.testing.assert_array_equal(v0, va)
    bad = make(kind, 300, 4, 7, seed=53, val_dtype=np.float32, gamma=0.95)
    if kind == "dense":
        bad.P = bad.P.copy(); bad.P[0, 0, :] *= 2.0
    else:
        bad.val = bad.val.copy(); bad.val[0, 0, :] *= 2.0
    keep3 = load(h1, bad, True)
    with pytest.raises(mg.MDPError) as e:
        mg.ipi_solve(h1, o)
    assert e.value.code == -1
    keep4 = load(h1, b, True)                  # the handle recovers with valid data
    v2, _, st2 = mg.ipi_solve(h1, o)
    np.testing.assert_array_equal(v2, v_ref)
    del keep, keep1, keep2, keep3, keep4


def test_iteration_cap_reports_noconv(mg):
    syn = make("ell", 200, 3, 4, seed=6, gamma=0.99)
    h = mg.from_synth(syn)
    v, pi, st = mg.vi_solve(h, mg.opts(tol=1e-12, precision="fp64", max_outer=3))
    assert st["status"] == -3 and st["outer"] == 3
    assert np.all(np.isfinite(v))


# ------------------------------------------------------------------ banded growth-model MDPs

@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_ipi_banded_ell_scaled(mg, prec):
    """Config-3-shaped MDP (banded columns around s + shift(a), quadratic costs) at S=6000,
    gamma=0.999, against the oracle's PI (dense LU)."""
    syn = mdp_synth.ell_banded(6000, 16, 32, 512, 64, 0.999, seed=1003,
                               val_dtype=np.float32 if prec == "mixed" else np.float64)
    m = oracle.from_synth(syn)
    ref = oracle.policy_iteration(m, tol=1e-11)
    h = mg.from_synth(syn)
    tol = 1e-8 if prec == "mixed" else 1e-11
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=tol, precision=prec))
    assert st["status"] == 0, st
    assert rel_err(v, ref.v) <= (1e-6 if prec == "mixed" else 1e-10)
    check_policy(pi, oracle.bellman(m, ref.v))


# ------------------------------------------------------------------ banded data: windowed sweep
# Columns within d.span of their state select the sweep that keeps a window of v in shared
# memory (spans up to 1792 states); the last case's span exceeds it and takes the global-gather
# sweep.  S spans one to many 256-state steps with ragged ends.
@pytest.mark.parametrize("S,hw,shift", [(1024, 8, 2), (1500, 100, 20), (4100, 512, 64),
                                        (16500, 1000, 100), (9000, 1700, 10), (9000, 1800, 10)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bellman_banded_window_parity(mg, S, hw, shift, prec):
    syn = mdp_synth.ell_banded(S, 6, 8, hw, shift, 0.99, seed=S + hw,
                               val_dtype=np.float32 if prec == "mixed" else np.float64)
    m = oracle.from_synth(syn)
    h = mg.from_synth(syn)
    rng = np.random.default_rng(S)
    for trial in range(2):
        v = rng.normal(size=S) * (10.0 if trial else 1.0) + 3.0 * trial
        sw = oracle.bellman(m, v)
        Tv, pi, res = mg.bellman_apply(h, v, precision=prec)
        tol = 1e-13 if prec == "fp64" else 1e-12
        assert rel_err(Tv, sw.Tv) <= tol
        assert abs(res - sw.res_inf) <= tol * max(1.0, np.max(np.abs(sw.Tv)))
        check_policy(pi, sw)
    h.close()


# Lane layouts of the windowed sweep (and of the bank order applied at upload to banded rows):
# A = 20 with 32 entries per row runs two passes per state at two lanes per row; A = 3 packs
# four states into a warp pass (each half-warp of the bank order spans two states); k = 16
# (one lane per row, 16 gather instructions) and k = 20 (20 instructions: rows keep their
# stored order) close the set.  Ragged S, a solve on the same handle, and a handle built from
# device arrays (the same bank order) give the same bits.
@pytest.mark.parametrize("S,A,k", [(5003, 20, 32), (4099, 3, 32), (3001, 7, 16), (2050, 5, 20)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_banded_window_lane_layouts(mg, S, A, k, prec):
    syn = mdp_synth.ell_banded(S, A, k, 400, 30, 0.99, seed=S + A,
                               val_dtype=np.float32 if prec == "mixed" else np.float64)
    m = oracle.from_synth(syn)
    h = mg.from_synth(syn)
    rng = np.random.default_rng(S + k)
    v = rng.normal(size=S) * 5.0
    sw = oracle.bellman(m, v)
    Tv, pi, res = mg.bellman_apply(h, v, precision=prec)
    tol = 1e-13 if prec == "fp64" else 1e-12
    assert rel_err(Tv, sw.Tv) <= tol
    assert abs(res - sw.res_inf) <= tol * max(1.0, np.max(np.abs(sw.Tv)))
    check_policy(pi, sw)
    vs, pis, st = mg.ipi_solve(h, mg.opts(tol=1e-9, precision=prec))
    assert st["status"] == 0
    h2 = mg.from_synth(syn, device=True)
    Tv2, pi2, res2 = mg.bellman_apply(h2, v, precision=prec)
    np.testing.assert_array_equal(np.asarray(Tv2), np.asarray(Tv))
    np.testing.assert_array_equal(np.asarray(pi2), np.asarray(pi))
    h.close()
    h2.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_windowed_and_global_sweeps_solve_alike(mg, prec):
    """The windowed sweep gathers the same v values as the global one, so per-state outputs
    agree bit for bit; only the grid's partial sums of ||Phi||_2 are grouped differently."""
    syn = mdp_synth.ell_banded(6000, 16, 32, 512, 64, 0.999, seed=1003,
                               val_dtype=np.float32 if prec == "mixed" else np.float64)
    h = mg.from_synth(syn)
    tol = 1e-9 if prec == "mixed" else 1e-11
    v1, pi1, st1 = mg.ipi_solve(h, mg.opts(tol=tol, precision=prec))
    v2, pi2, st2 = mg.ipi_solve(h, mg.opts(tol=tol, precision=prec, flags=mg.MDP_FLAG_NO_WINDOW))
    assert st1["status"] == 0 and st2["status"] == 0
    assert st1["outer"] == st2["outer"]
    assert rel_err(v1, v2) <= (1e-7 if prec == "mixed" else 1e-11)
    np.testing.assert_array_equal(pi1, pi2)
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_policy_sweeps_on_banded_data(mg, prec):
    """Policy sweeps (T^pi v, one row per state) also take the windowed kernel on banded data:
    OPI, Alg. 1 with VI inner steps and GMRES policy evaluation against the oracle."""
    syn = mdp_synth.ell_banded(5000, 8, 16, 300, 40, 0.95, seed=77,
                               val_dtype=np.float32 if prec == "mixed" else np.float64)
    m = oracle.from_synth(syn)
    ref = oracle.policy_iteration(m, tol=1e-12)
    h = mg.from_synth(syn)
    tol = 1e-8 if prec == "mixed" else 1e-11
    bound = 1e-6 if prec == "mixed" else 1e-9
    for solve in (mg.opi_solve, mg.ipi_vi_solve):
        v, pi, st = solve(h, mg.opts(tol=tol, precision=prec, opi_W=20, max_outer=2000))
        assert st["status"] == 0, (solve.__name__, st)
        assert rel_err(v, ref.v) <= bound
    pi0 = np.asarray(ref.pi, dtype=np.int32)
    ve, ste = mg.policy_eval_gmres(h, pi0, target_inf=1e-10, o=mg.opts(precision=prec))
    if prec == "fp64":
        assert ste["status"] == 0
        assert rel_err(ve, oracle.policy_evaluation(m, pi0)) <= 1e-10
    else:
        assert rel_err(ve, oracle.policy_evaluation(m, pi0)) <= 1e-6
    h.close()


def test_reload_changes_the_window_choice(mg):
    """A handle solved on banded data (windowed kernels, captured in the inner-loop graph) and
    then reloaded with uniformly spread columns of the same shape must switch back to the
    global-gather kernels: the solve of the new data matches the oracle."""
    S, A, k = 3000, 6, 16
    band = mdp_synth.ell_banded(S, A, k, 200, 30, 0.99, seed=11, val_dtype=np.float32)
    unif = mdp_synth.ell_uniform(S, A, k, 0.99, seed=12, val_dtype=np.float32)
    h = mg.from_synth(band)
    for syn in (band, unif, band):
        mg.mdp_load_ell(h, syn.col, syn.val, syn.g)
        m = oracle.from_synth(syn)
        ref = oracle.policy_iteration(m, tol=1e-11)
        v, pi, st = mg.ipi_solve(h, mg.opts(tol=1e-8, precision="mixed"))
        assert st["status"] == 0
        assert rel_err(v, ref.v) <= 1e-6
    h.close()


# ------------------------------------------------------------------ lucky breakdown
@pytest.mark.parametrize("kind", ["dense", "ell"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_absorbing_mdp_ends_every_inner_solve_by_lucky_breakdown(mg, kind, prec):
    """Every state absorbing (p_ss(a) = 1): J^pi = (1 - gamma) I, so the first Arnoldi vector
    spans an invariant Krylov space and the next direction vanishes: Alg. 2's breakdown branch
    ends each inner solve after one step with the exact least-squares solution.  v is the closed
    form min_a g(s, a) / (1 - gamma) and pi = argmin_a g(s, a)."""
    S, A, gamma = 37, 3, 0.95
    g = np.random.default_rng(4).random((A, S))
    vdt = np.float64 if prec == "fp64" else np.float32
    if kind == "dense":
        h = mg.mdp_create_dense(np.broadcast_to(np.eye(S, dtype=vdt), (A, S, S)).copy(), g, gamma)
    else:
        col = np.broadcast_to(np.arange(S, dtype=np.int32)[None, :, None], (A, S, 1)).copy()
        h = mg.mdp_create_ell(col, np.ones((A, S, 1), dtype=vdt), g, gamma)
    tol = 1e-12 if prec == "fp64" else 1e-9
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=tol, precision=prec))
    assert st["status"] == 0 and st["residual_inf"] <= tol
    # contraction bound: |v - v*| <= gamma * tol / (1 - gamma)
    np.testing.assert_allclose(v, g.min(0) / (1 - gamma), rtol=0,
                               atol=gamma * tol / (1 - gamma) + 1e-13)
    np.testing.assert_array_equal(pi, g.argmin(0))
    assert st["outer"] >= 1 and st["breakdowns"] == st["outer"] == st["inner"], st
    # policy evaluation alone reports the breakdown as informational success
    ve, ste = mg.policy_eval_gmres(h, g.argmin(0).astype(np.int32), target_inf=1e-10,
                                   o=mg.opts(precision=prec))
    assert ste["status"] == 1 and ste["breakdowns"] >= 1, ste
    # inverse bound: |V - V^pi| <= ||g - J V||_inf / (1 - gamma)
    np.testing.assert_allclose(ve, g.min(0) / (1 - gamma), rtol=0, atol=1e-10 / (1 - gamma))
    h.close()


# ------------------------------------------------------------------ bounded device waits
def test_bounded_wait_runs_out_and_the_context_stays_usable(mg):
    """A wait on an mbarrier that nothing completes, with a host-set limit of 2^20 cycles
    (about half a millisecond), returns MDP_ETIMEOUT through the same helper the bulk-copy
    pipelines use; the same wait with the arrival done returns MDP_OK; afterwards a dense sweep
    through the bulk-copy pipeline still matches the oracle."""
    lib = mg.lib()
    assert lib.mdp_selftest_wait(1 << 20, 0) == -5          # MDP_ETIMEOUT
    assert b"ran out" in lib.mdp_last_error()
    assert lib.mdp_selftest_wait(1 << 20, 1) == 0
    assert lib.mdp_selftest_wait(0, 0) == -1                # limit out of range: MDP_EINVAL
    syn = mdp_synth.dense_dirichlet(1200, 4, 0.1, 0.99, seed=3, dtype=np.float32)
    h = mg.from_synth(syn)
    v = np.random.default_rng(0).normal(size=syn.S) * 10
    sw = oracle.bellman(oracle.from_synth(syn), v)
    Tv, pi, res = mg.bellman_apply(h, v, precision="mixed")
    assert rel_err(Tv, sw.Tv) <= 1e-12
    check_policy(pi, sw)
    h.close()


def test_allocation_failure_reports_enomem_and_the_device_stays_usable(mg):
    """An MDP far larger than the device (2^31 - 65 states, 16 actions, 32 entries a row: about
    4.4 TB of values) fails in its first device allocation with MDP_ENOMEM, before any input is
    read (the inputs here are small placeholder buffers), and the next handle works."""
    import ctypes
    import torch
    lib = mg.lib()
    dummy = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    h = ctypes.c_void_p()
    S = (1 << 31) - 65
    rc = lib.mdp_create_ell_dev(S, 16, 32, p, p, mg.MDP_F32, p, 0.9, None, ctypes.byref(h))
    assert rc == -2 and not h.value                         # MDP_ENOMEM, no handle
    assert b"cudaMalloc" in lib.mdp_last_error()
    syn = make("ell", 300, 4, 7, seed=2, val_dtype=np.float32)
    hh = mg.from_synth(syn)
    v = np.random.default_rng(1).normal(size=300)
    sw = oracle.bellman(oracle.from_synth(syn), v)
    Tv, pi, res = mg.bellman_apply(hh, v, precision="mixed")
    assert rel_err(Tv, sw.Tv) <= 1e-12
    hh.close()
