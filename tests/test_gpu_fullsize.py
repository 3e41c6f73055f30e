"""Full-size parity on the benchmark workloads, element by element, through the C ABI.

Every state of every result is checked, in the launch configurations bench.py times:
  * config 2 (dense S=10^4, A=8, gamma=0.99): the whole v of the mixed solve (1e-6 relative)
    and of the plain FP64 solve at the tightened tolerance of reading A13 (1e-10 relative)
    against the oracle's Alg. 2 run to 1e-13; policies against the oracle's;
  * config 3 (banded S=10^6, A=16, k=32, gamma=0.999), plain and two-level preconditioned,
    whole v against the oracle's preconditioned Alg. 2 run to 1e-9;
  * config 4 (256 uneven ELL MDPs in one batch) in the mixed form and in the plain per-instance
    FP64 form;
  * config 5 (requests of the serving distribution at full size) through the serving loop.
Each result is certified by one FP64 oracle sweep at the returned v (tests/certify.py: the
residual bound gamma*r, the contraction bound on |v - V*| at every state, and the greedy policy
wherever its margin exceeds what the stopping tolerance can move), and the library's own Bellman
sweep at that v is compared with the oracle's sweep state by state (Tv 1e-12 relative in
double-float, 1e-13 in FP64; policies bit-exact where the oracle's two best Q-values differ by
more than 1e-9 relative).
"""
import numpy as np
import pytest

import mdp_synth
import oracle

from tests.certify import certify_solution, check_sweep

pytestmark = pytest.mark.gpu

TOL, ALPHA, W = 1e-8, 0.1, 30


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


def policy_against_reference(pi, ref, res_gpu, gamma):
    """The GPU's greedy policy at its V_K against the oracle's at its own V_K: both iterates lie
    within (r + r_ref) / (1 - gamma) of each other (contraction bound), which moves a Q-value by
    at most gamma times that; pi must agree wherever the oracle's margin exceeds twice the move
    (and the 1e-9 relative rule)."""
    move = gamma * (res_gpu + ref.residual) / (1.0 - gamma)
    q1 = np.abs(ref.v)
    thr = np.maximum(1e-9 * np.maximum(1.0, q1), 2.0 * move * (1 + 1e-9))
    sure = ref.margin > thr
    assert np.array_equal(np.asarray(pi)[sure], ref.pi[sure])
    return int(sure.sum())


# ------------------------------------------------------------------ config 2
@pytest.fixture(scope="module")
def cfg2():
    syn = mdp_synth.config(2)
    m = oracle.from_synth(syn)
    ref = oracle.gmres_policy_iteration(m, alpha=ALPHA, W=W, tol=1e-13)
    assert ref.status == "ok" and ref.residual <= 1e-13
    return syn, m, ref


def test_config2_mixed_whole_vector(mg, cfg2):
    syn, m, ref = cfg2
    h = mg.from_synth(syn)
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=TOL, alpha=ALPHA, restart=W, precision="mixed"))
    assert st["status"] == 0 and st["residual_inf"] <= TOL, st
    assert rel_err(v, ref.v) <= 1e-6
    policy_against_reference(pi, ref, st["residual_inf"], syn.gamma)
    sw, bound = certify_solution(m, v, pi, st["residual_inf"], 1e-6)
    Tv, pis, res = mg.bellman_apply(h, v, precision="mixed")
    check_sweep(sw, Tv, pis, res, 1e-12)
    h.close()


def test_config2_fp64_plain_whole_vector(mg, cfg2):
    """The plain FP64 form (P widened exactly, FP64 Krylov vectors and sums), solved to the
    tightened tolerance of reading A13: gamma * tol / (1 - gamma) <= 1e-10 * max|v| / 2."""
    syn, m, ref = cfg2
    syn64 = mdp_synth.SynthMDP(S=syn.S, A=syn.A, gamma=syn.gamma, g=syn.g, kind="dense",
                               P=syn.P.astype(np.float64))
    h = mg.from_synth(syn64)
    del syn64
    tol = 1e-10 * float(np.max(np.abs(ref.v))) * (1 - syn.gamma) / (2 * syn.gamma)
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=tol, alpha=ALPHA, restart=W, precision="fp64"))
    assert st["status"] == 0 and st["residual_inf"] <= tol, st
    assert rel_err(v, ref.v) <= 1e-10
    n_sure = policy_against_reference(pi, ref, st["residual_inf"], syn.gamma)
    assert n_sure >= 0.9 * syn.S
    sw, _ = certify_solution(m, v, pi, st["residual_inf"], 1e-10)
    Tv, pis, res = mg.bellman_apply(h, v, precision="fp64")
    check_sweep(sw, Tv, pis, res, 1e-13)
    h.close()


# ------------------------------------------------------------------ config 3
@pytest.fixture(scope="module")
def cfg3(mg):
    """The oracle's own solve of config 3: Alg. 2 with the two-level preconditioned inner
    GMRES (blocks of 512; plain Alg. 2 needs thousands of MGS steps at gamma = 0.999), to
    ||T v - v|| <= 1e-9, so that its values are within 1e-6 absolute of V*."""
    syn = mdp_synth.config(3)
    m = oracle.from_synth(syn)
    ref = oracle.gmres_policy_iteration(m, alpha=ALPHA, W=W, tol=1e-9, precond_block=512)
    assert ref.status == "ok"
    return syn, m, mg.from_synth(syn), ref


def test_config3_every_state(mg, cfg3):
    """S=10^6 banded, gamma=0.999, mixed: plain Alg. 2 and the two-level preconditioned inner
    solve with blocks of 512 states (the bench's two forms); the preconditioned solve also
    needs at least 4x fewer Arnoldi steps."""
    syn, m, h, ref = cfg3
    inner = {}
    for pb in (0, 512):
        v, pi, st = mg.ipi_solve(h, mg.opts(tol=TOL, alpha=ALPHA, restart=W, precision="mixed",
                                            precond_block=pb))
        assert st["status"] == 0 and st["residual_inf"] <= TOL, (pb, st)
        assert rel_err(v, ref.v) <= 1e-6
        policy_against_reference(pi, ref, st["residual_inf"], syn.gamma)
        sw, _ = certify_solution(m, v, pi, st["residual_inf"], 1e-6)
        Tv, pis, res = mg.bellman_apply(h, v, precision="mixed")
        check_sweep(sw, Tv, pis, res, 1e-12)
        inner[pb] = st["inner"]
        del sw
    assert inner[512] * 4 <= inner[0], inner


# ------------------------------------------------------------------ config 4
@pytest.fixture(scope="module")
def cfg4(mg):
    specs = mdp_synth.batch_specs(256, mdp_synth.CONFIG_SEEDS[4])
    syns = [mdp_synth.instance_from_spec(sp) for sp in specs]
    return syns, [mg.from_synth(s) for s in syns]


def test_config4_batch_every_instance_every_state(mg, cfg4):
    syns, hs = cfg4
    b = mg.MDPBatch(hs, mg.opts(tol=TOL, alpha=ALPHA, restart=W, precision="mixed"))
    b.tune()
    vs, ps, sts, code = b.solve()
    assert code == 0
    for syn, h, v, pi, st in zip(syns, hs, vs, ps, sts):
        assert st["status"] == 0 and st["residual_inf"] <= TOL, st
        m = oracle.from_synth(syn)
        sw, _ = certify_solution(m, v, pi, st["residual_inf"], 1e-6)
        Tv, pis, res = mg.bellman_apply(h, v, precision="mixed")
        check_sweep(sw, Tv, pis, res, 1e-12)
    b.close()


def test_config4_fp64_plain_per_instance(mg, cfg4):
    """The plain per-instance FP64 form on the same 256 MDPs (values widened exactly), each at
    its tightened tolerance: 1e-10 relative at every state."""
    syns, _ = cfg4
    for syn in syns:
        syn64 = mdp_synth.SynthMDP(S=syn.S, A=syn.A, gamma=syn.gamma, g=syn.g, kind="ell",
                                   col=syn.col, val=syn.val.astype(np.float64))
        h = mg.from_synth(syn64)
        m = oracle.from_synth(syn)
        v, pi, st = mg.ipi_solve(h, mg.opts(tol=TOL, alpha=ALPHA, restart=W, precision="fp64"))
        assert st["status"] == 0 and st["residual_inf"] <= TOL, st
        g = syn.gamma
        tol = 1e-10 * max(1.0, float(np.max(np.abs(v)))) * (1 - g) / (2 * g)
        v, pi, st = mg.ipi_solve(h, mg.opts(tol=tol, alpha=ALPHA, restart=W, precision="fp64",
                                            v0=v))
        assert st["status"] == 0 and st["residual_inf"] <= tol, st
        certify_solution(m, v, pi, st["residual_inf"], 1e-10)
        h.close()


# ------------------------------------------------------------------ config 5
def test_config5_served_requests_every_state(mg):
    """The first 24 distinct request MDPs of the serving trace at full size (S up to 2e5),
    submitted at once to the serving loop (continuous batching, HBM budget 120 GB)."""
    trace = mdp_synth.serving_trace(200.0, 60.0, mdp_synth.CONFIG_SEEDS[5])
    syns = [mdp_synth.instance_from_spec(sp) for sp in trace[:24]]
    srv = mg.MDPServer(o=mg.opts(tol=TOL, alpha=ALPHA, restart=W, precision="mixed"),
                       hbm_budget_bytes=120 << 30)
    ids = [srv.submit(np.ascontiguousarray(s.col), np.ascontiguousarray(s.val),
                      np.ascontiguousarray(s.g), s.gamma) for s in syns]
    got = {rid: (v, pi, st) for rid, v, pi, st in srv.drain()}
    srv.close()
    assert sorted(got) == sorted(ids)
    for rid, syn in zip(ids, syns):
        v, pi, st = got[rid]
        assert st["status"] == 0 and st["residual_inf"] <= TOL, st
        certify_solution(oracle.from_synth(syn), v, pi, st["residual_inf"], 1e-6)
