"""Sharding bank 2 across ranks: per-shard searches merged with renumbered
sequences equal the unsharded search byte for byte (the oracle stands in for
each rank's GPU); the two-rank version gathers over gloo."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_0804_3643_gb300 import shard, synth


def search(b1, codes, seq_off):
    o1 = oracle.make_bank(b1.codes, b1.seq_off)
    o2 = oracle.make_bank(codes, seq_off)
    return oracle.small_gapped(o1, o2, oracle.ungapped(o1, o2, threads=4))


@pytest.fixture(scope="module")
def banks():
    return synth.workload("plastp_plain", seed=6, scale=0.3)


def test_ranges_cover_the_bank():
    rng = np.random.default_rng(0)
    for n, world in [(1, 1), (5, 3), (40, 4), (3, 8), (0, 2)]:
        off = np.zeros(n + 1, dtype=np.int64)
        off[1:] = np.cumsum(rng.integers(0, 50, n))
        ranges = [shard.shard_range(off, r, world) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        assert all(a[1] == b[0] and a[0] <= a[1] for a, b in zip(ranges, ranges[1:]))
    with pytest.raises(ValueError):
        shard.shard_range(np.zeros(3, np.int64), 2, 2)


@pytest.mark.parametrize("world", [2, 3])
def test_merged_shards_equal_unsharded(banks, world):
    b1, b2 = banks
    want = search(b1, b2.codes, b2.seq_off)
    assert len(want) > 20
    parts = []
    for r in range(world):
        c, o, first = shard.shard_bank(b2.codes, b2.seq_off, r, world)
        parts.append((search(b1, c, o), first))
    got = shard.merge_records(parts)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8))


def test_merged_shard_alignments_equal_unsharded(banks):
    # stage 3.2 per shard: a pair of sequences lies in one shard, so its
    # redundancy list does too
    b1, b2 = banks
    o1 = oracle.make_bank(b1.codes, b1.seq_off)
    want = oracle.full_gapped(o1, oracle.make_bank(b2.codes, b2.seq_off), search(b1, b2.codes, b2.seq_off))
    assert len(want) > 10
    parts = []
    for r in range(3):
        c, o, first = shard.shard_bank(b2.codes, b2.seq_off, r, 3)
        parts.append((oracle.full_gapped(o1, oracle.make_bank(c, o), search(b1, c, o)), first))
    got = shard.merge_records(parts)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle as orc
    from paper_0804_3643_gb300 import shard as sh, synth as sy

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    b1, b2 = sy.workload("plastp_plain", seed=6, scale=0.3)
    c, o, first = sh.shard_bank(b2.codes, b2.seq_off, rank, world)
    o1 = orc.make_bank(b1.codes, b1.seq_off)
    o2 = orc.make_bank(c, o)
    recs = orc.small_gapped(o1, o2, orc.ungapped(o1, o2, threads=2))
    parts = [None] * world
    dist.all_gather_object(parts, (recs.tobytes(), first))
    if rank == 0:
        dt = recs.dtype
        merged = sh.merge_records([(np.frombuffer(b, dtype=dt), f) for b, f in parts])
        out["merged"] = merged.tobytes()
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gather_and_merge(banks):
    b1, b2 = banks
    want = search(b1, b2.codes, b2.seq_off)
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        got = out["merged"]
    assert got == want.tobytes()
