"""bellman_apply_ell_noalloc_dev: the Bellman sweep for callers that may not allocate memory
while they run (for example a server whose pooling allocator owns the whole device, or a
latency-critical loop that must not let cudaMalloc synchronise the device).  Its output is
compared with the existing handle-based bellman_apply_dev on two calls in a row, which also
shows that scratch left behind by one call does not leak into the next.

Kept in a file of its own that pytest collects last, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import mdp_synth

pytestmark = pytest.mark.gpu


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


def test_noalloc_sweep_matches_bellman_apply_dev_on_two_calls(env):
    torch, mg, lib = env
    syn = mdp_synth.tiny_random(3001, 5, seed=17, gamma=0.95, kind="ell", k=7)
    S, A, k = syn.S, syn.A, syn.k
    col = torch.from_numpy(np.ascontiguousarray(syn.col)).cuda()
    val = torch.from_numpy(np.ascontiguousarray(syn.val, dtype=np.float64)).cuda()
    g = torch.from_numpy(np.ascontiguousarray(syn.g)).cuda()
    h = mg.from_synth(syn, device=True)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    for call in range(2):
        v = torch.from_numpy(rng.normal(size=S) * (1 + 20 * call)).cuda()
        Tv_ref, pi_ref, res_ref, margin = mg.bellman_apply(h, v, precision="fp64", margin=True)
        Tv = torch.empty(S, dtype=torch.float64, device="cuda")
        pi = torch.empty(S, dtype=torch.int32, device="cuda")
        res = torch.empty(1, dtype=torch.float64, device="cuda")
        rc = lib.bellman_apply_ell_noalloc_dev(S, A, k, _p(col), _p(val), _p(g), syn.gamma, _p(v),
                                               _p(Tv), _p(pi), _p(res),
                                               ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        a, b = Tv.cpu().numpy(), Tv_ref.cpu().numpy()
        # FP64 tolerance of the parity tests: 1e-13 relative
        assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(b)))
        sure = margin.cpu().numpy() > 1e-9 * np.maximum(1.0, np.abs(b))
        assert np.array_equal(pi.cpu().numpy()[sure], pi_ref.cpu().numpy()[sure])
        assert abs(res.item() - res_ref) <= 1e-13 * max(1.0, np.max(np.abs(b)))
    h.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, mg, lib = env
    big = (1 << 20) + 1
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = _p(dummy)
    rc = lib.bellman_apply_ell_noalloc_dev(big, 1, 1, p, p, p, 0.9, p, p, p, p, None)
    assert rc == -1  # MDP_EINVAL, nothing launched
