"""CUDA path vs the oracle on the other workloads at their full sizes:

* batching stress: 50,000 x 50,000 proteins, 20 % with low-complexity runs
  (heavy-tailed key lists, 5.4e10 pairs);
* TPLAST-N: 5,000 proteins vs 50 Mbp translated on the device (1e8 aa);
* PLAST-X: 1,000 sequences of about 1 kbp vs 50 Mbp, both translated on the
  device;
* serving: a 1,000,000-protein resident bank against a 250-protein query.

Each comparison runs the GPU on a random sample of keys (plast_ungapped_ex /
plast_search_ex with a key list, the per-key decomposition of Section 5.1) and requires the records to equal the
oracle's stages 1-3.1 over the same keys byte for byte.  The six-frame
translation is compared in full.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_0804_3643_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_0804_3643_gb300 import binding, build

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    binding.lib()
    binding.plast_set_schedule(0)
    return binding


def sample_keys(o1, o2, rng, n, lo=10 ** 4, hi=4 * 10 ** 6, budget=6 * 10 ** 7):
    pp = np.diff(o1.idx.key_off) * np.diff(o2.idx.key_off)
    cand = rng.permutation(np.nonzero((pp >= lo) & (pp <= hi))[0])
    keys, tot = [], 0
    for k in cand:
        if len(keys) >= n or tot + pp[k] > budget:
            continue
        keys.append(int(k))
        tot += int(pp[k])
    return np.sort(np.array(keys, dtype=np.int32)), tot


def check_keys(B, g1, g2, o1, o2, keys):
    want_h = oracle.ungapped(o1, o2, keys=keys, threads=16)
    got_h = B.hits_numpy(B.plast_ungapped_ex(g1, g2, keys=keys))
    assert np.array_equal(got_h.view(np.uint8), want_h.view(np.uint8))
    del got_h
    want_g = oracle.small_gapped(o1, o2, want_h, threads=16)
    recs, n_ung = B.plast_search_ex(g1, g2, keys=keys)
    assert n_ung == len(want_h)
    assert np.array_equal(B.gapped_numpy(recs).view(np.uint8), want_g.view(np.uint8))
    return len(want_h), len(want_g)


def test_batching_stress_full_size(B):
    b1, b2 = synth.workload("batching_stress", seed=1)
    d1 = B.DeviceBank.from_host(b1.codes, b1.seq_off)
    d2 = B.DeviceBank.from_host(b2.codes, b2.seq_off)
    g1 = B.plast_index_bank(d1.codes, d1.seq_off)
    g2 = B.plast_index_bank(d2.codes, d2.seq_off)
    o1 = oracle.make_bank(b1.codes, b1.seq_off)
    o2 = oracle.make_bank(b2.codes, b2.seq_off)
    assert B.plast_pair_count(g1, g2) > 5 * 10 ** 10
    keys, pairs = sample_keys(o1, o2, np.random.default_rng(31), 40)
    # low-complexity keys: the three with the most pairs (about 2e8 each, up
    # to 45 million stage-2 hits per key), the lists the persistent queue cuts
    # across tiles and CTAs, plus three with 4e6 to 2e7 pairs
    pp = np.diff(o1.idx.key_off) * np.diff(o2.idx.key_off)
    order = np.argsort(pp)[::-1]
    top = order[:3]
    assert pp[top].min() > 10 ** 8
    mid = order[(pp[order] > 4 * 10 ** 6) & (pp[order] < 2 * 10 ** 7)][:3]
    keys = np.unique(np.concatenate([keys, top.astype(np.int32), mid.astype(np.int32)]))
    nh, ng = check_keys(B, g1, g2, o1, o2, keys)
    assert nh > 10 ** 7 and ng > 10 ** 6
    try:
        B.plast_set_schedule(1)
        r1, _ = B.plast_search_ex(g1, g2, keys=keys)
    finally:
        B.plast_set_schedule(0)
    r0, _ = B.plast_search_ex(g1, g2, keys=keys)
    assert np.array_equal(r0.cpu().numpy(), r1.cpu().numpy())


def test_tplastn_full_size(B):
    b1, dna = synth.tplastn_workload(seed=1)
    aa, so, meta = B.plast_translate6(torch.from_numpy(dna.codes).cuda(), torch.from_numpy(dna.seq_off).cuda())
    w_aa, w_so, w_meta = oracle.translate6(dna.codes, dna.seq_off)
    assert len(w_aa) > 9 * 10 ** 7
    assert np.array_equal(aa.cpu().numpy(), w_aa)
    assert np.array_equal(so.cpu().numpy(), w_so)
    assert np.array_equal(meta.cpu().numpy(), w_meta)
    d1 = B.DeviceBank.from_host(b1.codes, b1.seq_off)
    g1 = B.plast_index_bank(d1.codes, d1.seq_off)
    g2 = B.plast_index_bank(aa, so)
    o1 = oracle.make_bank(b1.codes, b1.seq_off)
    o2 = oracle.make_bank(w_aa, w_so)
    keys, _ = sample_keys(o1, o2, np.random.default_rng(32), 40)
    nh, ng = check_keys(B, g1, g2, o1, o2, keys)
    assert nh > 1000


def test_plastx_full_size(B):
    q, subj = synth.plastx_workload(seed=1)
    banks = []
    for dna in (q, subj):
        aa, so, meta = B.plast_translate6(torch.from_numpy(dna.codes).cuda(), torch.from_numpy(dna.seq_off).cuda())
        w_aa, w_so, w_meta = oracle.translate6(dna.codes, dna.seq_off)
        assert np.array_equal(aa.cpu().numpy(), w_aa)
        assert np.array_equal(so.cpu().numpy(), w_so)
        assert np.array_equal(meta.cpu().numpy(), w_meta)
        banks.append((B.plast_index_bank(aa, so), oracle.make_bank(w_aa, w_so)))
    (g1, o1), (g2, o2) = banks
    assert B.plast_pair_count(g1, g2) > 10 ** 10
    keys, _ = sample_keys(o1, o2, np.random.default_rng(33), 40)
    nh, ng = check_keys(B, g1, g2, o1, o2, keys)
    assert nh > 1000


def test_serving_resident_bank_full_size(B):
    rng = np.random.default_rng(1)
    bank = synth.random_protein_bank(rng, 1_000_000)
    q = synth.random_protein_bank(np.random.default_rng(33), 250)
    dq = B.DeviceBank.from_host(q.codes, q.seq_off)
    db = B.DeviceBank.from_host(bank.codes, bank.seq_off)
    gq = B.plast_index_bank(dq.codes, dq.seq_off)
    gb = B.plast_index_bank(db.codes, db.seq_off)
    oq = oracle.make_bank(q.codes, q.seq_off)
    ob = oracle.make_bank(bank.codes, bank.seq_off)
    keys, _ = sample_keys(oq, ob, np.random.default_rng(34), 60, lo=10 ** 3)
    nh, ng = check_keys(B, gq, gb, oq, ob, keys)
    assert nh > 100
