"""Batched iGMRES-PI (mdp_batch_* / ipi_solve_batch) on the GPU, through the C ABI.

Each instance of a batch runs Alg. 2 with the same kernel bodies as a single solve; only the
block geometry (which fixes the order of floating-point additions) is the batch's own.  So:
  * against the oracle: values within 1e-6 relative at ||T(v)-v||_inf <= 1e-8 (mixed path),
    policies bit-exact where the oracle's margin is clear (same rule as the single solves);
  * against ipi_solve on the same handle with the batch's lanes and block counts: equal bit
    for bit, with the same outer and inner iteration counts;
  * an instance's result does not depend on the other instances of its batch.
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


def scaled_specs(n, seed, scale):
    out = []
    for sp in mdp_synth.batch_specs(n, seed):
        sp = dict(sp)
        sp["S"] = max(sp["k"] + 1, int(sp["S"] * scale))
        out.append(sp)
    return out


def handles_for(mg, specs):
    syns = [mdp_synth.instance_from_spec(sp) for sp in specs]
    return syns, [mg.from_synth(s) for s in syns]


OPTS = dict(tol=1e-8, precision="mixed", alpha=0.1, restart=30)


def test_batch_matches_oracle_scaled(mg):
    """16 instances of the batched workload's distribution, S scaled by 1/20 (25..2500),
    against the oracle's PI (dense LU evaluation)."""
    specs = scaled_specs(16, 1004, 0.05)
    syns, hs = handles_for(mg, specs)
    b = mg.MDPBatch(hs, mg.opts(**OPTS))
    vs, ps, sts, code = b.solve()
    assert code == 0
    for syn, v, pi, st in zip(syns, vs, ps, sts):
        assert st["status"] == 0 and st["residual_inf"] <= 1e-8, st
        m = oracle.from_synth(syn)
        ref = oracle.policy_iteration(m, tol=1e-11)
        assert rel_err(v, ref.v) <= 1e-6
        check_policy(pi, oracle.bellman(m, ref.v))
        # certified by the oracle's own Bellman step at the returned v
        assert oracle.bellman(m, v).res_inf <= syn.gamma * 1e-8 * 1.01 + 1e-12


def _alone_equal(mg, b, hs, vs, ps, sts):
    for i, h in enumerate(hs):
        g = b.geometry(i)
        h.set_tuning(g["lanes_sweep"], g["lanes_matvec"])
        h.set_geometry(g["sweep_blocks"], g["matvec_blocks"], g["krylov_blocks"])
        v, pi, st = mg.ipi_solve(h, mg.opts(**OPTS))
        np.testing.assert_array_equal(v, vs[i])
        np.testing.assert_array_equal(pi, ps[i])
        assert (st["outer"], st["inner"], st["status"]) == \
            (sts[i]["outer"], sts[i]["inner"], sts[i]["status"])
        h.set_tuning(0, 0)
        h.set_geometry(0, 0, 0)


def test_batch_equals_single_solves_bitwise(mg):
    specs = scaled_specs(10, 2024, 0.2)
    _, hs = handles_for(mg, specs)
    b = mg.MDPBatch(hs, mg.opts(**OPTS))
    vs, ps, sts, code = b.solve()
    assert code == 0
    _alone_equal(mg, b, hs, vs, ps, sts)


def test_batch_tuned_equals_single_solves_bitwise(mg):
    specs = scaled_specs(12, 7, 0.3)
    _, hs = handles_for(mg, specs)
    b = mg.MDPBatch(hs, mg.opts(**OPTS))
    b.tune()
    lanes = {(b.geometry(i)["lanes_sweep"], b.geometry(i)["lanes_matvec"]) for i in range(len(hs))}
    assert all(ls in (1, 2, 4, 8) and lm in (1, 2, 4, 8) for ls, lm in lanes)
    vs, ps, sts, code = b.solve()
    assert code == 0
    _alone_equal(mg, b, hs, vs, ps, sts)


def test_batch_composition_does_not_matter(mg):
    specs = scaled_specs(9, 99, 0.1)
    _, hs = handles_for(mg, specs)
    full = mg.MDPBatch(hs, mg.opts(**OPTS))
    vs, ps, sts, _ = full.solve()
    sub_idx = [7, 2, 4]
    sub = mg.MDPBatch([hs[i] for i in sub_idx], mg.opts(**OPTS))
    vs2, ps2, sts2, _ = sub.solve()
    for j, i in enumerate(sub_idx):
        np.testing.assert_array_equal(vs2[j], vs[i])
        np.testing.assert_array_equal(ps2[j], ps[i])
        assert sts2[j]["inner"] == sts[i]["inner"]


def test_batch_device_outputs_and_replay(mg):
    import torch
    specs = scaled_specs(6, 5, 0.1)
    _, hs = handles_for(mg, specs)
    b = mg.MDPBatch(hs, mg.opts(**OPTS))
    vs, ps, sts, _ = b.solve()
    vd, pd, sts_d, code = b.solve(device=True)
    assert code == 0
    for i in range(len(hs)):
        np.testing.assert_array_equal(vd[i].cpu().numpy(), vs[i])
        np.testing.assert_array_equal(pd[i].cpu().numpy(), ps[i])
    # a second replay of the same graph gives the same results
    vs3, ps3, _, _ = b.solve()
    for i in range(len(hs)):
        np.testing.assert_array_equal(vs3[i], vs[i])
    torch.cuda.synchronize()


def test_one_shot_equals_batch_object(mg):
    specs = scaled_specs(5, 11, 0.05)
    _, hs = handles_for(mg, specs)
    vs, ps, sts, code = mg.ipi_solve_batch(hs, mg.opts(**OPTS))
    b = mg.MDPBatch(hs, mg.opts(**OPTS))
    vs2, ps2, _, _ = b.solve()
    assert code == 0
    for i in range(len(hs)):
        np.testing.assert_array_equal(vs[i], vs2[i])
        np.testing.assert_array_equal(ps[i], ps2[i])


def test_batch_masks_single_action_and_tiny_states(mg):
    """Masked actions, A = 1, S = 1 and k = S instances in one batch, against brute force
    (tiny) or the oracle's PI."""
    syns = [mdp_synth.tiny_random(3, 2, seed=1, gamma=0.9, kind="ell", k=2, mask_frac=0.0,
                                  val_dtype=np.float32),
            mdp_synth.tiny_random(1, 3, seed=2, gamma=0.95, kind="ell", k=1,
                                  val_dtype=np.float32),
            mdp_synth.tiny_random(300, 1, seed=3, gamma=0.99, kind="ell", k=5,
                                  val_dtype=np.float32),
            mdp_synth.tiny_random(400, 6, seed=4, gamma=0.999, kind="ell", k=9, mask_frac=0.4,
                                  val_dtype=np.float32),
            mdp_synth.tiny_random(4, 3, seed=8, gamma=0.9, kind="ell", k=4, mask_frac=0.3,
                                  val_dtype=np.float32)]
    hs = [mg.from_synth(s) for s in syns]
    vs, ps, sts, code = mg.MDPBatch(hs, mg.opts(**OPTS)).solve()
    assert code == 0
    for syn, v, pi, st in zip(syns, vs, ps, sts):
        m = oracle.from_synth(syn)
        ref_v = oracle.brute_force(m)[0] if syn.S <= 4 and syn.A <= 3 else \
            oracle.policy_iteration(m, tol=1e-12).v
        assert st["status"] == 0
        assert rel_err(v, ref_v) <= 1e-6
        check_policy(pi, oracle.bellman(m, ref_v))


def test_batch_iteration_cap(mg):
    specs = scaled_specs(4, 3, 0.05)
    syns, hs = handles_for(mg, specs)
    b = mg.MDPBatch(hs, mg.opts(tol=1e-14, precision="mixed", max_outer=1))
    vs, ps, sts, code = b.solve()
    assert code == -3
    for syn, v, pi, st in zip(syns, vs, ps, sts):
        assert st["status"] == -3 and st["outer"] == 1
        assert np.all(np.isfinite(v)) and np.all((pi >= 0) & (pi < syn.A))


def test_batch_rejects_invalid_inputs(mg):
    ell64 = mdp_synth.tiny_random(50, 3, seed=1, kind="ell", k=4, val_dtype=np.float64)
    dense = mdp_synth.tiny_random(50, 3, seed=1, kind="dense", val_dtype=np.float32)
    ok = mdp_synth.tiny_random(50, 3, seed=1, kind="ell", k=4, val_dtype=np.float32)
    h64, hd, hok = mg.from_synth(ell64), mg.from_synth(dense), mg.from_synth(ok)
    for hs in ([h64], [hd], [hok, hd]):
        with pytest.raises(mg.MDPError) as e:
            mg.MDPBatch(hs, mg.opts(**OPTS))
        assert e.value.code == -1
    for bad in (dict(precision="fp64"), dict(alpha=0.0), dict(restart=65),
                dict(v0=np.zeros(50))):
        kw = dict(OPTS)
        kw.update(bad)
        with pytest.raises(mg.MDPError) as e:
            mg.MDPBatch([hok], mg.opts(**kw))
        assert e.value.code == -1


def test_host_loop_equals_graph_and_batched_bellman(mg):
    """The host-driven loop runs the same kernels as the graph (results equal bit for bit);
    the batched Bellman sweep at the final V_K reproduces each instance's ||Phi_K||_inf."""
    specs = scaled_specs(7, 13, 0.1)
    syns, hs = handles_for(mg, specs)
    vs, ps, sts, _ = mg.MDPBatch(hs, mg.opts(**OPTS)).solve()
    hb = mg.MDPBatch(hs, mg.opts(flags=mg.MDP_FLAG_HOST_LOOP, **OPTS))
    vs2, ps2, sts2, code = hb.solve()
    assert code == 0
    for i in range(len(hs)):
        np.testing.assert_array_equal(vs2[i], vs[i])
        np.testing.assert_array_equal(ps2[i], ps[i])
        assert sts2[i]["inner"] == sts[i]["inner"]
    res = hb.bellman()
    np.testing.assert_array_equal(res, [s["residual_inf"] for s in sts2])
    for syn, v, r in zip(syns, vs2, res):
        m = oracle.from_synth(syn)
        # v = T(V_K): the oracle's residual at v is at most gamma * ||Phi_K||_inf (contraction)
        assert oracle.bellman(m, v).res_inf <= syn.gamma * r * 1.01 + 1e-12
