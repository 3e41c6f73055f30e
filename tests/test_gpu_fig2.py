"""GMRES vs VI for policy evaluation across gamma at n = 100 states (the study of Fig. 2, Sec. 3.1).

With one action per state every policy is the same, VI is policy evaluation (T = T^pi) and the
paper's claim is about this setting: the Arnoldi steps GMRES needs to reach a residual hardly
change with gamma (the eigenvalues of I - gamma P^pi cluster in the disc of the spectrum
lemma), while VI needs about log(tol) / log(gamma) sweeps.  The GPU counts must equal the
oracle's (VI exactly, up to one sweep at the threshold; GMRES within two Arnoldi steps, the
GPU orthogonalises by CGS2 and the oracle by MGS).
"""
import numpy as np
import pytest

import mdp_synth
import oracle

pytestmark = pytest.mark.gpu

GAMMAS = (0.5, 0.9, 0.99, 0.999)
TARGET = 1e-8


@pytest.fixture(scope="module")
def mg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_04299_gb300 import build
    build.build()
    import paper_2211_04299_gb300 as mg
    return mg


def test_fig2_gmres_robust_to_gamma_vi_not(mg):
    rows = []
    for g in GAMMAS:
        syn = mdp_synth.dense_dirichlet(100, 1, 1.0, g, seed=2022, dtype=np.float64)
        m = oracle.from_synth(syn)
        pi0 = np.zeros(100, np.int32)
        ref_g = oracle.policy_eval_gmres(m, pi0, target_inf=TARGET, W=64)
        ref_v = oracle.value_iteration(m, tol=TARGET, max_iter=10 ** 6)
        h = mg.from_synth(syn)
        v_g, st_g = mg.policy_eval_gmres(h, pi0, target_inf=TARGET,
                                         o=mg.opts(precision="fp64", restart=64))
        v_v, _, st_v = mg.vi_solve(h, mg.opts(precision="fp64", tol=TARGET, max_outer=10 ** 6))
        h.close()
        assert st_g["status"] == 0 and st_v["status"] == 0
        vstar = oracle.policy_evaluation(m, pi0)
        scale = max(1.0, float(np.max(np.abs(vstar))))
        assert np.max(np.abs(v_g - vstar)) <= 2 * TARGET / (1 - g) + 1e-12 * scale
        assert np.max(np.abs(v_v - vstar)) <= 2 * TARGET / (1 - g) + 1e-12 * scale
        assert abs(st_v["outer"] - ref_v.outer) <= 1, (g, st_v["outer"], ref_v.outer)
        assert abs(st_g["inner"] - ref_g.inner) <= 2, (g, st_g["inner"], ref_g.inner)
        rows.append((g, st_g["inner"], st_v["outer"]))
    print("gamma  GMRES steps  VI sweeps:", rows)
    g_steps = [r[1] for r in rows]
    v_sweeps = [r[2] for r in rows]
    # VI follows log(tol)/log(gamma); GMRES barely moves across three orders of 1/(1-gamma)
    assert v_sweeps[-1] >= 100 * v_sweeps[0]
    assert g_steps[-1] <= 2 * g_steps[0] + 2
    assert all(s <= 100 for s in g_steps)
