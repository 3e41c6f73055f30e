"""Exchange layer of the row-sharded solve on CPU: gloo ranks call the host collectives
through the same C function pointers the library calls (mdp_comm.allgather / allreduce), on
ragged row partitions; no GPU and no kernel is involved."""
import ctypes
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, S, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import paper_2211_04299_gb300 as mg
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rb = mg.row_partition(S, world)
    comm = mg.ShardComm(rb)
    lo, hi = int(rb[rank]), int(rb[rank + 1])
    local = (np.arange(lo, hi, dtype=np.float64) * 1.5 + 0.25)
    glob = np.full(S, np.nan)
    rc1 = comm.c.allgather(None, local.ctypes.data, glob.ctypes.data, 8)
    vals = np.array([rank + 1.0, -2.0 * rank, 0.5], dtype=np.float64)
    p = vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc2 = comm.c.allreduce(None, p, 3, 0)
    summed = vals.copy()
    vals[:] = [rank + 1.0, -2.0 * rank, 0.5]
    rc3 = comm.c.allreduce(None, p, 3, 1)
    maxed = vals.copy()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, rc1, rc2, rc3, glob, summed, maxed))


@pytest.mark.parametrize("world,S", [(2, 7), (3, 10), (3, 3)])
def test_host_collectives_through_the_c_callbacks(world, S):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, S, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ranks = np.arange(world)
    for rank, rc1, rc2, rc3, glob, summed, maxed in out:
        assert rc1 == rc2 == rc3 == 0
        np.testing.assert_array_equal(glob, np.arange(S) * 1.5 + 0.25)
        np.testing.assert_array_equal(summed, [np.sum(ranks + 1.0), np.sum(-2.0 * ranks), 0.5 * world])
        np.testing.assert_array_equal(maxed, [world, 0.0, 0.5])


def test_row_partition_is_contiguous_and_balanced():
    sys.path.insert(0, ROOT)
    import paper_2211_04299_gb300 as mg
    for S, world in [(10, 3), (2000, 7), (5, 5), (1, 1)]:
        rb = mg.row_partition(S, world)
        assert rb[0] == 0 and rb[-1] == S and np.all(np.diff(rb) >= 0)
        assert np.max(np.diff(rb)) - np.min(np.diff(rb)) <= 1
