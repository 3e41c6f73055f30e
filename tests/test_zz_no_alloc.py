"""bellman_apply_ell_noalloc_dev: the Bellman sweep for callers that may not allocate memory
while they run (for example a server whose pooling allocator owns the whole device, or a
latency-critical loop that must not let cudaMalloc synchronise the device).

Its outputs are compared with the oracle's FP64 Bellman sweep (Sec. 2) and with the existing
handle-based bellman_apply_dev on several calls in a row whose sizes shrink, so that scratch
left behind by a larger call cannot leak into a smaller one; a call with a column index out of
range must report NaN and the next clean call must be exact again (the flag it raised is
cleared).  Tolerance: the FP64 parity tests' 1e-13 relative.

Kept in a file of its own that pytest collects last, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import mdp_synth
import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_04299_gb300 import build
    build.build()
    import paper_2211_04299_gb300 as mg
    return torch, mg, mg.lib()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _call(torch, lib, syn, col_np, v_np, stream):
    S, A, k = syn.S, syn.A, syn.k
    col = torch.from_numpy(np.ascontiguousarray(col_np)).cuda()
    val = torch.from_numpy(np.ascontiguousarray(syn.val, dtype=np.float64)).cuda()
    g = torch.from_numpy(np.ascontiguousarray(syn.g)).cuda()
    v = torch.from_numpy(np.ascontiguousarray(v_np)).cuda()
    Tv = torch.full((S,), -7.0, dtype=torch.float64, device="cuda")
    pi = torch.full((S,), -1, dtype=torch.int32, device="cuda")
    res = torch.full((1,), -7.0, dtype=torch.float64, device="cuda")
    rc = lib.bellman_apply_ell_noalloc_dev(S, A, k, _p(col), _p(val), _p(g), syn.gamma, _p(v),
                                           _p(Tv), _p(pi), _p(res),
                                           ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc, Tv.cpu().numpy(), pi.cpu().numpy(), res.item()


def _check(sw, Tv, pi, res):
    scale = max(1.0, float(np.max(np.abs(sw.Tv))))
    assert float(np.max(np.abs(Tv - sw.Tv))) <= TOL * scale
    assert abs(res - sw.res_inf) <= TOL * scale
    q1 = sw.Q[sw.pi, np.arange(sw.Q.shape[1])]
    sure = sw.margin > 1e-9 * np.maximum(1.0, np.abs(q1))
    assert np.array_equal(pi[sure], sw.pi[sure])


def test_noalloc_sweep_matches_oracle_and_bellman_apply_dev_on_calls_in_a_row(env):
    torch, mg, lib = env
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    # shrinking sizes: 12 blocks of scratch maxima, then 6, then 1 (a ragged 1-block grid)
    for call, S in enumerate((3001, 1500, 200)):
        syn = mdp_synth.tiny_random(S, 5, seed=17 + call, gamma=0.95, kind="ell", k=7)
        v = rng.normal(size=S) * (1 + 20 * call)
        rc, Tv, pi, res = _call(torch, lib, syn, syn.col, v, stream)
        assert rc == 0
        sw = oracle.bellman(oracle.from_synth(syn), v)
        _check(sw, Tv, pi, res)
        h = mg.from_synth(syn, device=True)
        Tv_ref, pi_ref, res_ref = mg.bellman_apply(h, torch.from_numpy(v).cuda(), precision="fp64")
        h.close()
        np.testing.assert_allclose(Tv, Tv_ref.cpu().numpy(), rtol=0, atol=TOL * max(1.0, np.max(np.abs(Tv))))
        assert abs(res - res_ref) <= TOL * max(1.0, np.max(np.abs(Tv)))


def test_noalloc_reports_bad_columns_then_recovers(env):
    torch, mg, lib = env
    stream = torch.cuda.current_stream()
    syn = mdp_synth.tiny_random(700, 3, seed=23, gamma=0.9, kind="ell", k=5)
    v = np.random.default_rng(2).normal(size=syn.S)
    bad = syn.col.copy()
    bad[1, 345, 2] = syn.S          # one column index out of range: skipped, reported as NaN
    rc, Tv, pi, res = _call(torch, lib, syn, bad, v, stream)
    assert rc == 0 and np.isnan(res)
    assert np.all(np.isfinite(Tv)) and np.all((pi >= 0) & (pi < syn.A))
    # the next call on the same stream starts from a cleared flag and is exact again
    rc, Tv, pi, res = _call(torch, lib, syn, syn.col, v, stream)
    assert rc == 0 and np.isfinite(res)
    _check(oracle.bellman(oracle.from_synth(syn), v), Tv, pi, res)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, mg, lib = env
    big = (1 << 20) + 1
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = _p(dummy)
    rc = lib.bellman_apply_ell_noalloc_dev(big, 1, 1, p, p, p, 0.9, p, p, p, p, None)
    assert rc == -1  # MDP_EINVAL, nothing launched
