"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): each rank
draws its own bank-2 shard, the job's time is the slowest rank's, and the
whole-job rate counts every rank's units.  No data-path collective exists;
only this timing reduction."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_0804_3643_gb300 import synth

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank
    out[rank] = (bench.reduce_max(ms, world, "cpu"), bench.shard_seed(rank))
    _, b2 = synth.workload("plastp_plain", seed=bench.shard_seed(rank), scale=0.01)
    out[world + rank] = int(b2.codes.astype(np.int64).sum())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_shards():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0       # both ranks see the slowest rank's time
    assert res[0][1] != res[1][1]                 # distinct shard seeds
    assert res[2] != res[3]                       # distinct bank-2 shards
    import bench
    assert bench.whole_job_rate(1e9, 2, 150.0) == 2e9 / 0.15
