"""Multi-rank host logic of the frame-sharded batch path, as world_size-2 gloo ranks on CPU:
the ranks' frame sets are disjoint and cover the batch, and the job time is the maximum over
ranks (no data-path collective exists to test)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_frames, out):
    import torch
    import torch.distributed as dist
    from paper_2505_03932_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.frames_for_rank(n_frames, rank, world)
    flags = torch.zeros(n_frames, dtype=torch.int64)
    flags[mine] = 1
    dist.all_reduce(flags)  # coverage check only; the reprojection itself exchanges nothing
    t = shard.max_over_ranks(1.5 + rank)
    out[rank] = (flags.tolist(), t, mine)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("n_frames", [64, 7, 1])
def test_frames_shard_over_two_gloo_ranks(n_frames):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, n_frames, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    flags0, t0, mine0 = res[0]
    flags1, t1, mine1 = res[1]
    assert flags0 == [1] * n_frames and flags1 == [1] * n_frames  # each frame exactly once
    assert not set(mine0) & set(mine1)
    assert t0 == t1 == 2.5  # the max over ranks
