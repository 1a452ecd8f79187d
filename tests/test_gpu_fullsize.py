"""CUDA path vs the oracle at the benchmark's full size (10,000 x 100,000
proteins, 2.15e10 pairs, in the launch configuration bench.py times).

The oracle cannot redo the whole comparison in seconds, so:
* for a random sample of keys, the GPU's stage-2 hits of those keys equal
  the oracle's stages 1-2 over the same keys, byte for byte, and the GPU's
  stage-3.1 records of those keys equal the oracle's stage 3.1 of them;
* a random sample of all stage-3.1 records is recomputed one by one;
* properties that hold at any size: canonical order, thresholds, records
  are a subset of the hits with the same ungapped score, both schedules
  (persistent queue and one launch per key) give identical output.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_0804_3643_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    from paper_0804_3643_gb300 import binding as B
    from paper_0804_3643_gb300 import build

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    B.lib()
    B.plast_set_schedule(0)
    b1, b2 = synth.workload("plastp_full", seed=1)
    d1 = B.DeviceBank.from_host(b1.codes, b1.seq_off)
    d2 = B.DeviceBank.from_host(b2.codes, b2.seq_off)
    g1 = B.plast_index_bank(d1.codes, d1.seq_off)
    g2 = B.plast_index_bank(d2.codes, d2.seq_off)
    hits = B.hits_numpy(B.plast_ungapped(g1, g2))
    recs_t, n_ung = B.plast_search_ex(g1, g2)
    recs = B.gapped_numpy(recs_t)
    o1 = oracle.make_bank(b1.codes, b1.seq_off)
    o2 = oracle.make_bank(b2.codes, b2.seq_off)
    return B, g1, g2, o1, o2, hits, recs, n_ung


def keys_of(o, seq, pos):
    """Subset-seed key of each word (seq, pos), from the oracle's class tables."""
    cls = np.array([[oracle.seed_class(p, a) for a in range(20)] for p in (1, 2, 3, 4)], dtype=np.int64)
    start = o.seq_off[seq] + pos
    w = [o.codes[start + t].astype(np.int64) for t in range(4)]
    return ((cls[0][w[0]] * 2 + cls[1][w[1]]) * 11 + cls[2][w[2]]) * 20 + cls[3][w[3]]


def sorted_canonically(a):
    k = np.stack([a["seq1"], a["pos1"], a["seq2"], a["pos2"]]).astype(np.int64)
    d = np.diff(k, axis=1)
    first = np.argmax(d != 0, axis=0)
    return bool((d[first, np.arange(d.shape[1])] > 0).all())


def test_fullsize_invariants(full):
    B, g1, g2, o1, o2, hits, recs, n_ung = full
    assert B.plast_pair_count(g1, g2) == int((np.diff(o1.idx.key_off) * np.diff(o2.idx.key_off)).sum())
    assert n_ung == len(hits) > 10 ** 7
    assert (hits["score"] >= 38).all() and (recs["score"] >= 47).all()
    assert sorted_canonically(hits) and sorted_canonically(recs)
    assert (recs["score"] >= recs["ungapped"]).all()
    # every record is a stage-2 hit with the same ungapped score
    hk = (hits["seq1"].astype(np.int64) << 40) | (hits["pos1"].astype(np.int64) << 30) | \
         (hits["seq2"].astype(np.int64) << 12) | hits["pos2"].astype(np.int64)
    rk = (recs["seq1"].astype(np.int64) << 40) | (recs["pos1"].astype(np.int64) << 30) | \
         (recs["seq2"].astype(np.int64) << 12) | recs["pos2"].astype(np.int64)
    at = np.searchsorted(hk, rk)
    assert (hk[at] == rk).all()
    assert (hits["score"][at] == recs["ungapped"]).all()


def test_fullsize_sampled_keys_bit_exact(full):
    B, g1, g2, o1, o2, hits, recs, n_ung = full
    n1 = np.diff(o1.idx.key_off)
    n2 = np.diff(o2.idx.key_off)
    rng = np.random.default_rng(17)
    cand = np.nonzero((n1 * n2 > 0) & (n1 * n2 < 3_000_000))[0]
    sample = np.sort(rng.choice(cand, size=24, replace=False))
    # the heaviest key too: its tiles run first on the persistent queue
    sample = np.unique(np.append(sample, np.argmax(n1 * n2)))
    want_h = oracle.ungapped(o1, o2, keys=sample, threads=8)
    hkeys = keys_of(o1, hits["seq1"], hits["pos1"])
    got_h = hits[np.isin(hkeys, sample)]
    assert len(want_h) > 1000
    assert np.array_equal(got_h.view(np.uint8), want_h.view(np.uint8))
    want_g = oracle.small_gapped(o1, o2, want_h, threads=16)
    rkeys = keys_of(o1, recs["seq1"], recs["pos1"])
    got_g = recs[np.isin(rkeys, sample)]
    assert np.array_equal(got_g.view(np.uint8), want_g.view(np.uint8))


def test_fullsize_sampled_records_one_by_one(full):
    B, g1, g2, o1, o2, hits, recs, n_ung = full
    rng = np.random.default_rng(5)
    for r in recs[rng.choice(len(recs), size=3000, replace=False)]:
        x = o1.codes[o1.seq_off[r["seq1"]]:o1.seq_off[r["seq1"] + 1]]
        y = o2.codes[o2.seq_off[r["seq2"]]:o2.seq_off[r["seq2"] + 1]]
        u = oracle.ungapped_pair(x, int(r["pos1"]), y, int(r["pos2"]))[0]
        g = oracle.small_gapped_pair(x, int(r["pos1"]), y, int(r["pos2"]))
        assert (int(r["ungapped"]), int(r["score"]), int(r["r_i"]), int(r["r_j"]), int(r["l_i"]), int(r["l_j"])) \
            == (u,) + g


def test_fullsize_schedules_agree(full):
    B, g1, g2, o1, o2, hits, recs, n_ung = full
    try:
        B.plast_set_schedule(1)
        r1, n1 = B.plast_search_ex(g1, g2)
    finally:
        B.plast_set_schedule(0)
    assert n1 == n_ung
    assert np.array_equal(B.gapped_numpy(r1).view(np.uint8), recs.view(np.uint8))
