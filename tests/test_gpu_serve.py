"""Serving loop (mdp_server_*): continuous batching through the C ABI, on the GPU.

Requests are admitted while others are solving and share every loop launch with them; each
slot's arithmetic is the batch engine's and never reads another slot, so every result must
equal, bit for bit, the same MDP solved alone by ipi_solve with the batch engine's kernel
shape (and by a one-instance batch), and match the oracle within the mixed-path tolerances
(values 1e-6 relative at ||T(v)-v||_inf <= 1e-8; policies bit-exact where the oracle's
margin is clear).
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


OPTS = dict(tol=1e-8, precision="mixed", alpha=0.1, restart=30)


def requests(n, seed, scale):
    """n request MDPs from the serving distribution (S log-uniform in [1e3, 2e5] scaled,
    A in {4, 8, 16}, k = 16, gamma in {0.95, 0.99}), FP32 values."""
    out = []
    for sp in mdp_synth.serving_trace(200.0, 60.0, seed)[:n]:
        sp = dict(sp)
        sp["S"] = max(sp["k"] + 1, int(sp["S"] * scale))
        out.append(mdp_synth.instance_from_spec(sp))
    return out


def alone(mg, syn):
    """ipi_solve of the MDP alone with the batch engine's kernel shape."""
    h = mg.from_synth(syn)
    g = mg.MDPBatch([h], mg.opts(**OPTS)).geometry(0)
    h.set_tuning(g["lanes_sweep"], g["lanes_matvec"])
    h.set_geometry(g["sweep_blocks"], g["matvec_blocks"], g["krylov_blocks"])
    v, pi, st = mg.ipi_solve(h, mg.opts(**OPTS))
    h.close()
    return v, pi, st


def submit(srv, syn):
    return srv.submit(np.ascontiguousarray(syn.col), np.ascontiguousarray(syn.val),
                      np.ascontiguousarray(syn.g), syn.gamma)


def test_requests_joining_a_running_mix_equal_alone(mg):
    syns = requests(8, 5, 0.05)
    srv = mg.MDPServer(o=mg.opts(**OPTS), iters_per_launch=2)
    ids = [submit(srv, s) for s in syns[:3]]
    got = {}
    for _ in range(6):                      # the first three are on the device ...
        for rid, v, pi, st in srv.poll():
            got[rid] = (v, pi, st)
    assert srv.info()["active"] > 0
    ids += [submit(srv, s) for s in syns[3:6]]   # ... when these arrive
    for _ in range(3):
        for rid, v, pi, st in srv.poll():
            got[rid] = (v, pi, st)
    ids += [submit(srv, s) for s in syns[6:]]
    for rid, v, pi, st in srv.drain():
        got[rid] = (v, pi, st)
    assert sorted(got) == sorted(ids)
    for rid, syn in zip(ids, syns):
        v, pi, st = got[rid]
        assert st["status"] == 0 and st["residual_inf"] <= 1e-8, st
        va, pa, sa = alone(mg, syn)
        np.testing.assert_array_equal(v, va)
        np.testing.assert_array_equal(pi, pa)
        assert (st["outer"], st["inner"]) == (sa["outer"], sa["inner"])
        assert st["seconds"] > 0


def test_served_results_match_oracle(mg):
    syns = requests(5, 17, 0.01)
    srv = mg.MDPServer(o=mg.opts(**OPTS))
    ids = [submit(srv, s) for s in syns]
    res = {rid: (v, pi, st) for rid, v, pi, st in srv.drain()}
    for rid, syn in zip(ids, syns):
        v, pi, st = res[rid]
        assert st["status"] == 0
        m = oracle.from_synth(syn)
        ref = oracle.policy_iteration(m, tol=1e-11)
        assert np.max(np.abs(v - ref.v)) / max(1.0, np.max(np.abs(ref.v))) <= 1e-6
        sw = oracle.bellman(m, ref.v)
        q1 = sw.Q.min(axis=0)
        sure = sw.margin > 1e-9 * np.maximum(1.0, np.abs(q1))
        assert np.array_equal(pi[sure], sw.pi[sure])


def test_budget_and_slots_queue_requests_without_changing_results(mg):
    syns = requests(6, 23, 0.03)
    free = mg.MDPServer(o=mg.opts(**OPTS))
    ids = [submit(free, s) for s in syns]
    ref = {rid: (v, pi) for rid, v, pi, _ in free.drain()}
    # a budget of about two requests and two slots: the others wait in the queue
    sizes = [s.S * s.A * 16 * 8 * 2 + s.S * 200 for s in syns]
    tight = mg.MDPServer(o=mg.opts(**OPTS), hbm_budget_bytes=2 * max(sizes) + (8 << 20),
                         max_slots=2)
    ids2 = [submit(tight, s) for s in syns]
    seen_pending = tight.info()["pending"] > 0
    got = {}
    while len(got) < len(syns):
        for rid, v, pi, st in tight.poll():
            assert st["status"] == 0, st
            got[rid] = (v, pi)
        info = tight.info()
        seen_pending |= info["pending"] > 0
        assert info["active"] <= 2
    assert seen_pending
    for a, b in zip(ids, ids2):
        np.testing.assert_array_equal(got[b][0], ref[a][0])
        np.testing.assert_array_equal(got[b][1], ref[a][1])


def test_invalid_and_oversized_requests_fail_alone(mg):
    good = requests(2, 31, 0.01)
    bad = requests(1, 37, 0.01)[0]
    bad.val = bad.val.copy()
    bad.val[0, 0, :] *= 2.0                    # a row that does not sum to 1
    srv = mg.MDPServer(o=mg.opts(**OPTS))
    ids = [submit(srv, good[0]), submit(srv, bad), submit(srv, good[1])]
    res = {rid: st for rid, _, _, st in srv.drain()}
    assert res[ids[0]]["status"] == 0 and res[ids[2]]["status"] == 0
    assert res[ids[1]]["status"] == -1
    small = mg.MDPServer(o=mg.opts(**OPTS), hbm_budget_bytes=4096)  # below any request
    rid = submit(small, good[0])
    res = {r: st for r, _, _, st in small.drain()}
    assert res[rid]["status"] == -2


def test_device_output_buffers(mg):
    import torch
    syn = requests(1, 41, 0.02)[0]
    srv = mg.MDPServer(o=mg.opts(**OPTS))
    vd = torch.empty(syn.S, dtype=torch.float64, device="cuda")
    pd = torch.empty(syn.S, dtype=torch.int32, device="cuda")
    srv.submit(np.ascontiguousarray(syn.col), np.ascontiguousarray(syn.val),
               np.ascontiguousarray(syn.g), syn.gamma, v_out=vd, pi_out=pd)
    (rid, v, pi, st), = srv.drain()
    va, pa, _ = alone(mg, syn)
    np.testing.assert_array_equal(vd.cpu().numpy(), va)
    np.testing.assert_array_equal(pd.cpu().numpy(), pa)
