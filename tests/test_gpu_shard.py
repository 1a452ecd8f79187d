"""Sharded search on the GPU: bank 2 cut into sequence ranges, each searched
with plast_search (as each rank would on its own GPU), the records merged:
equal to the unsharded plast_search and to the oracle; the same with stage
3.2 run per shard and the alignments merged."""
import numpy as np
import pytest
import torch

import oracle
from paper_0804_3643_gb300 import shard, synth

pytestmark = pytest.mark.gpu


def test_sharded_search_merges_to_the_full_search():
    from paper_0804_3643_gb300 import binding as B, build

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    b1, b2 = synth.workload("plastp_plain", seed=12, scale=0.5)
    d1 = B.DeviceBank.from_host(b1.codes, b1.seq_off)
    g1 = B.plast_index_bank(d1.codes, d1.seq_off)

    def search(codes, seq_off, full_gapped=False):
        d = B.DeviceBank.from_host(codes, seq_off)
        g = B.plast_index_bank(d.codes, d.seq_off)
        recs, _ = B.plast_search_ex(g1, g)
        if full_gapped:
            return B.alignments_numpy(B.plast_full_gapped(g1, g, recs)[0]).copy()
        return B.gapped_numpy(recs).copy()

    full = search(b2.codes, b2.seq_off)
    o1, o2 = oracle.make_bank(b1.codes, b1.seq_off), oracle.make_bank(b2.codes, b2.seq_off)
    want = oracle.small_gapped(o1, o2, oracle.ungapped(o1, o2, threads=16))
    assert np.array_equal(full.view(np.uint8), want.view(np.uint8))
    for world in (2, 4):
        parts = []
        for r in range(world):
            c, o, first = shard.shard_bank(b2.codes, b2.seq_off, r, world)
            parts.append((search(c, o), first))
        merged = shard.merge_records(parts)
        assert np.array_equal(merged.view(np.uint8), full.view(np.uint8))
    # stage 3.2 per shard, the alignments merged: equal to stage 3.2 of the
    # full search and to the oracle's
    full_al = search(b2.codes, b2.seq_off, full_gapped=True)
    assert np.array_equal(full_al.view(np.uint8), oracle.full_gapped(o1, o2, want, threads=16).view(np.uint8))
    for world in (2, 4):
        parts = []
        for r in range(world):
            c, o, first = shard.shard_bank(b2.codes, b2.seq_off, r, world)
            parts.append((search(c, o, full_gapped=True), first))
        assert np.array_equal(shard.merge_records(parts).view(np.uint8), full_al.view(np.uint8))
