"""Adaptive forcing sequence (mdp_opts.forcing_c) on the GPU against the oracle.

alpha_k = min(alpha, c ||Phi_k||_inf) with the inner threshold kept >= tol / 10 (Sec. 3 local
convergence theorem: Q-superlinear when alpha_k -> 0).  The GPU computes the same threshold
expression as the oracle's inner_threshold; results must match the oracle at the usual
tolerances (FP64 1e-10 relative with tol tightened as in the config-1 test, mixed 1e-6), and
the batch must still equal single solves bit for bit.
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
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(1.0, float(np.max(np.abs(b)))))


def test_fp64_adaptive_forcing_matches_oracle(mg):
    syn = mdp_synth.config(1)                      # ELL S=2000, A=5, k=16, gamma=0.95, FP64
    m = oracle.from_synth(syn)
    ref = oracle.gmres_policy_iteration(m, alpha=0.1, W=30, tol=1e-13, forcing_c=1.0)
    h = mg.from_synth(syn)
    tol = 1e-10 * np.max(np.abs(ref.v)) * (1 - 0.95) / (2 * 0.95)
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=tol, precision="fp64", forcing_c=1.0))
    _, _, st0 = mg.ipi_solve(h, mg.opts(tol=tol, precision="fp64"))
    assert st["status"] == 0 and st["residual_inf"] <= tol
    assert rel_err(v, ref.v) <= 1e-10
    assert st["outer"] <= st0["outer"]            # alpha_k <= alpha never needs more outer steps here


def test_mixed_adaptive_forcing_matches_oracle(mg):
    syn = mdp_synth.config(1)
    syn.val = syn.val.astype(np.float32)
    m = oracle.from_synth(syn)
    ref = oracle.gmres_policy_iteration(m, alpha=0.1, W=30, tol=1e-13, forcing_c=1.0)
    h = mg.from_synth(syn)
    v, pi, st = mg.ipi_solve(h, mg.opts(tol=1e-8, precision="mixed", forcing_c=1.0))
    assert st["status"] == 0 and st["residual_inf"] <= 1e-8
    assert rel_err(v, ref.v) <= 1e-6
    assert oracle.bellman(m, v).res_inf <= 0.95e-8 * 1.01


def test_batch_with_forcing_equals_single_solves(mg):
    specs = mdp_synth.batch_specs(6, 77)
    hs = []
    for sp in specs:
        sp = dict(sp)
        sp["S"] = max(sp["k"] + 1, sp["S"] // 10)
        hs.append(mg.from_synth(mdp_synth.instance_from_spec(sp)))
    o = dict(tol=1e-8, precision="mixed", forcing_c=2.0)
    b = mg.MDPBatch(hs, mg.opts(**o))
    vs, ps, sts, code = b.solve()
    assert code == 0
    for i, h in enumerate(hs):
        g = b.geometry(i)
        h.set_tuning(g["lanes_sweep"], g["lanes_matvec"])
        h.set_geometry(g["sweep_blocks"], g["matvec_blocks"], g["krylov_blocks"])
        v, pi, st = mg.ipi_solve(h, mg.opts(**o))
        np.testing.assert_array_equal(v, vs[i])
        np.testing.assert_array_equal(pi, ps[i])
        assert st["outer"] == sts[i]["outer"] and st["inner"] == sts[i]["inner"]
