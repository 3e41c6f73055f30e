"""Row-sharded iGMRES-PI (ipi_solve_sharded) against the oracle, on the GPU.

World sizes 2 and 3 run as gloo processes that share this one GPU: every exchange is a host
collective between kernel launches and no kernel waits on another rank, so the ranks need not
run at the same time.  Each rank creates its rows of the MDP (contiguous balanced blocks, the
last ragged), solves, and returns its slice of v = T(V_K) and pi; the gathered vector must meet
the FP64 path's tolerance (1e-10 relative, with tol tightened as in reading A13) against the
oracle's Alg. 2 run to 1e-13, and pi must match wherever the oracle's margin is clear.  Every
rank reports the same outer / inner counts (the replicated Givens state takes the same
decisions everywhere).  Banded columns cross the shard boundaries, uniform ones reach every
shard."""
import os
import socket
import sys

import numpy as np
import pytest

import mdp_synth
import oracle

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _make(kind, vdt):
    if kind == "uniform":
        return mdp_synth.ell_uniform(2000, 5, 16, 0.95, seed=1001, val_dtype=vdt)
    return mdp_synth.ell_banded(3000, 6, 16, 120, 25, 0.99, seed=77, val_dtype=vdt)


def _rank_main(rank, world, port, kind, vdt, tol, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    try:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(0)
        import paper_2211_04299_gb300 as mg
        dist.init_process_group("gloo", rank=rank, world_size=world)
        syn = _make(kind, vdt)
        rb = mg.row_partition(syn.S, world)
        lo, hi = int(rb[rank]), int(rb[rank + 1])
        h = mg.mdp_shard_create(syn.S, lo, syn.col[:, lo:hi], syn.val[:, lo:hi], syn.g[:, lo:hi],
                                syn.gamma)
        comm = mg.ShardComm(rb)
        v, pi, st = mg.ipi_solve_sharded(h, comm, mg.opts(tol=tol, alpha=0.1, restart=30))
        h.close()
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, lo, v, pi, st, None))
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, 0, None, None, None, repr(e)))


def _run(world, kind, vdt, tol):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, kind, vdt, tol, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=600) for _ in procs], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
    errs = [x[5] for x in out if x[5]]
    assert not errs, errs
    assert all(p.exitcode == 0 for p in procs)
    return out


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("kind", ["uniform", "banded"])
@pytest.mark.parametrize("vdt", [np.float64, np.float32])
def test_sharded_solve_matches_oracle(world, kind, vdt):
    syn = _make(kind, vdt)
    m = oracle.from_synth(syn)
    ref = oracle.gmres_policy_iteration(m, alpha=0.1, W=30, tol=1e-13)
    g = syn.gamma
    tol = 1e-10 * float(np.max(np.abs(ref.v))) * (1 - g) / (2 * g)
    out = _run(world, kind, vdt, tol)
    v = np.concatenate([x[2] for x in out])
    pi = np.concatenate([x[3] for x in out])
    sts = [x[4] for x in out]
    for st in sts:
        assert st["status"] == 0 and st["residual_inf"] <= tol, st
        assert (st["outer"], st["inner"], st["restarts"]) == \
            (sts[0]["outer"], sts[0]["inner"], sts[0]["restarts"])
    assert float(np.max(np.abs(v - ref.v)) / np.max(np.abs(ref.v))) <= 1e-10
    sw = oracle.bellman(m, ref.v)
    q1 = np.min(sw.Q, axis=0)
    sure = sw.margin > 1e-9 * np.maximum(1.0, np.abs(q1))
    assert np.array_equal(pi[sure], sw.pi[sure])
    # the contraction bound certifies every state of the gathered v
    assert oracle.bellman(m, v).res_inf <= g * tol + 1e-12 * np.max(np.abs(v))


def _mismatch_main(port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK="0", WORLD_SIZE="1")
    sys.path.insert(0, ROOT)
    try:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(0)
        import paper_2211_04299_gb300 as mg
        dist.init_process_group("gloo", rank=0, world_size=1)
        syn = _make("uniform", np.float64)
        h = mg.mdp_shard_create(syn.S, 0, syn.col, syn.val, syn.g, syn.gamma)
        codes = []
        for rb in ([0, syn.S - 1], [0, syn.S + 1]):   # partitions that do not match the shard
            try:
                mg.ipi_solve_sharded(h, mg.ShardComm(np.array(rb)), mg.opts())
                codes.append(0)
            except mg.MDPError as e:
                codes.append(e.code)
        v, pi, st = mg.ipi_solve_sharded(h, mg.ShardComm(mg.row_partition(syn.S, 1)),
                                         mg.opts(tol=1e-10, precision="fp64"))
        bad_col = syn.col.copy()
        bad_col[0, 5, 0] = syn.S
        try:
            mg.mdp_shard_create(syn.S, 0, bad_col, syn.val, syn.g, syn.gamma)
            codes.append(0)
        except mg.MDPError as e:
            codes.append(e.code)
        h.close()
        dist.destroy_process_group()
        q.put((codes, v, st, None))
    except Exception as e:
        q.put((None, None, None, repr(e)))


def test_sharded_solve_rejects_a_mismatched_partition_and_runs_on_one_rank():
    """A communicator whose row partition does not match the shard is rejected (MDP_EINVAL)
    before any exchange, as is a column index outside [0, S); one rank owning every row solves
    to the oracle's values."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_mismatch_main, args=(_free_port(), q))
    p.start()
    codes, v, st, err = q.get(timeout=600)
    p.join(timeout=120)
    assert err is None, err
    assert codes == [-1, -1, -1]
    syn = _make("uniform", np.float64)
    ref = oracle.gmres_policy_iteration(oracle.from_synth(syn), alpha=0.1, W=30, tol=1e-13)
    assert st["status"] == 0
    assert float(np.max(np.abs(v - ref.v)) / np.max(np.abs(ref.v))) <= 1e-10
