"""CUDA path vs the CPU oracle, through the C ABI, element by element.

Integer work throughout, so the bar is bit-exact: the same index, the same
hit set with the same scores and extents, the same small gapped records in
the same canonical order.
"""
import numpy as np
import pytest
import torch

import oracle
from conftest import bank_from
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


def gpu_bank(B, codes, seq_off):
    d = B.DeviceBank.from_host(codes, seq_off)
    return B.plast_index_bank(d.codes, d.seq_off)


def both(B, codes, seq_off):
    return gpu_bank(B, codes, seq_off), oracle.make_bank(codes, seq_off)


def same(a: np.ndarray, b: np.ndarray) -> bool:
    return a.shape == b.shape and np.array_equal(a.view(np.uint8), b.view(np.uint8))


def check_index(B, g, o):
    key_off, pos = B.plast_bank_export_index(g)
    assert np.array_equal(key_off.cpu().numpy(), o.idx.key_off)
    assert np.array_equal(pos.cpu().numpy(), o.idx.pos)


@pytest.fixture(scope="module")
def plain(B):
    b1, b2 = synth.workload("plastp_plain", seed=1)
    g1, o1 = both(B, b1.codes, b1.seq_off)
    g2, o2 = both(B, b2.codes, b2.seq_off)
    return g1, o1, g2, o2


def test_index_parity(B, plain):
    g1, o1, g2, o2 = plain
    check_index(B, g1, o1)
    check_index(B, g2, o2)


def test_index_edge_banks(B):
    cases = [
        ["AQAA"],                        # one word
        ["AQA", "W", ""],                # no word at all
        ["", "", "MKVLAAQAAWWW", ""],    # empty sequences around
        ["A" * 300, "AQAASAAAPAAA" * 20],  # long lists of one key
        ["MKV*LAQ*AAAA*", "**AQAA**"],  # stops are never inside an indexed word
    ]
    for seqs in cases:
        c, o = bank_from(seqs)
        g, ob = both(B, c, o)
        check_index(B, g, ob)


def test_index_many_tiles_low_complexity(B):
    # a bank cut into many index tiles, with low-complexity runs (keys repeated
    # many times within one warp's 32 positions and across tile borders)
    _, b2 = synth.workload("batching_stress", seed=5, scale=0.05)
    g, o = both(B, b2.codes, b2.seq_off)
    assert len(b2.codes) > 500_000
    check_index(B, g, o)


def test_ungapped_parity_plain(B, plain):
    g1, o1, g2, o2 = plain
    got = B.hits_numpy(B.plast_ungapped(g1, g2))
    want = oracle.ungapped(o1, o2)
    assert len(want) > 1000
    assert same(got, want)


def test_search_parity_plain(B, plain):
    g1, o1, g2, o2 = plain
    recs, n_ung = B.plast_search_ex(g1, g2)
    want_h = oracle.ungapped(o1, o2)
    want = oracle.small_gapped(o1, o2, want_h)
    assert n_ung == len(want_h)
    assert len(want) > 100
    assert same(B.gapped_numpy(recs), want)


def test_small_gapped_on_given_hits(B, plain):
    g1, o1, g2, o2 = plain
    hits = oracle.ungapped(o1, o2, oracle.Params(s1=30))
    prm = oracle.Params(s2=-10 ** 4)
    want = oracle.small_gapped(o1, o2, hits, prm)
    got = B.plast_small_gapped(g1, g2, B.hits_from_numpy(hits), B.plast_default_params(s2=-10 ** 4))
    assert len(want) == len(hits)
    assert same(B.gapped_numpy(got), want)


def test_thresholds_and_gap_costs(B, plain):
    g1, o1, g2, o2 = plain
    # the edges of the gap costs the int16 row offsets allow: no gap cost at
    # all, free opening, costly opening, the largest extension
    for s1, s2, go, ge in [(25, 30, 11, 1), (45, 60, 10, 2), (38, 47, 5, 3), (38, 47, 0, 0), (38, 47, 0, 4),
                           (38, 40, 1000, 1), (38, 40, 7, 400)]:
        prm = oracle.Params(s1=s1, s2=s2, gap_open=go, gap_extend=ge)
        gp = B.plast_default_params(s1=s1, s2=s2, gap_open=go, gap_extend=ge)
        recs, n_ung = B.plast_search_ex(g1, g2, gp)
        want_h = oracle.ungapped(o1, o2, prm)
        assert n_ung == len(want_h)
        assert same(B.gapped_numpy(recs), oracle.small_gapped(o1, o2, want_h, prm))


def test_ungapped_threshold_range_edges(B, plain):
    # S1 at the ends of its range: the stage-2 kernels find the hit rows from
    # the sign of m - S1 in int16, which stays exact from -30000 to 30000
    g1, o1, g2, o2 = plain
    for s1 in (30000, 29, -30000):
        got = B.hits_numpy(B.plast_ungapped(g1, g2, B.plast_default_params(s1=s1)))
        want = oracle.ungapped(o1, o2, oracle.Params(s1=s1))
        assert same(got, want), s1
        if s1 == 30000:
            assert len(want) == 0
        if s1 == -30000:
            assert len(want) == B.plast_pair_count(g1, g2)  # every pair


def test_gap_cost_limits(B, plain):
    g1, _, g2, _ = plain
    for go, ge in [(1001, 1), (11, 401), (-1, 1), (11, -1)]:
        with pytest.raises(B.PlastError):
            B.plast_search(g1, g2, B.plast_default_params(gap_open=go, gap_extend=ge))


def test_plain_schedule_matches_persistent(B):
    b1, b2 = synth.workload("plastp_plain", seed=2, scale=0.3)
    g1, o1 = both(B, b1.codes, b1.seq_off)
    g2, o2 = both(B, b2.codes, b2.seq_off)
    want = oracle.ungapped(o1, o2)
    try:
        B.plast_set_schedule(1)
        per_key = B.hits_numpy(B.plast_ungapped(g1, g2))
    finally:
        B.plast_set_schedule(0)
    persistent = B.hits_numpy(B.plast_ungapped(g1, g2))
    assert same(per_key, want) and same(persistent, want)


def test_identical_banks_every_pair_passes(B):
    # self comparison with S1 = 0: every pair passes, so per-warp buffers
    # overflow and the direct-write path runs
    rng = np.random.default_rng(3)
    seqs = [rng.integers(0, 4, int(rng.integers(20, 200))).astype(np.int8) for _ in range(30)]
    c, o = bank_from(seqs)
    g, ob = both(B, c, o)
    # a search at the default S1 first: the survivor buffer of the pair's
    # next search is sized from its (low) rate, so the S1 = 0 searches below
    # overflow it and take the run with the exact count
    recs, _ = B.plast_search_ex(g, g)
    w_hits = oracle.ungapped(ob, ob)
    assert same(B.gapped_numpy(recs), oracle.small_gapped(ob, ob, w_hits))
    prm = oracle.Params(s1=0, s2=-10 ** 4)
    want = oracle.ungapped(ob, ob, prm)
    got = B.hits_numpy(B.plast_ungapped(g, g, B.plast_default_params(s1=0)))
    assert len(want) == oracle.ungapped(ob, ob, prm, return_pairs=True)[1]
    assert same(got, want)
    w_recs = oracle.small_gapped(ob, ob, want, prm)
    for _ in range(2):  # the second sized from the first's rate and count
        recs, _ = B.plast_search_ex(g, g, B.plast_default_params(s1=0, s2=-10 ** 4))
        assert same(B.gapped_numpy(recs), w_recs)


def test_low_complexity_workload(B):
    b1, b2 = synth.workload("batching_stress", seed=4, scale=0.004)
    g1, o1 = both(B, b1.codes, b1.seq_off)
    g2, o2 = both(B, b2.codes, b2.seq_off)
    want = oracle.ungapped(o1, o2, threads=8)
    got = B.hits_numpy(B.plast_ungapped(g1, g2))
    assert same(got, want)
    recs, _ = B.plast_search_ex(g1, g2)
    assert same(B.gapped_numpy(recs), oracle.small_gapped(o1, o2, want))


def test_empty_and_tiny_banks(B):
    c0, o0 = bank_from([])
    c1, o1 = bank_from(["AQAA"])
    c2, o2 = bank_from(["AQAAW", "SQAAC"])
    e = gpu_bank(B, c0, o0)
    a = gpu_bank(B, c1, o1)
    b = gpu_bank(B, c2, o2)
    assert B.plast_ungapped(e, a).shape[0] == 0
    assert B.plast_ungapped(a, e).shape[0] == 0
    h = B.hits_numpy(B.plast_ungapped(a, b, B.plast_default_params(s1=-100)))
    want = oracle.ungapped(oracle.make_bank(c1, o1), oracle.make_bank(c2, o2), oracle.Params(s1=-100))
    assert same(h, want) and len(want) == 1


def test_translate6_parity(B):
    rng = np.random.default_rng(9)
    lens = [0, 1, 2, 3, 5, 7, 30, 301, 1000, 1001, 1002]
    contigs = [rng.integers(0, 4, L).astype(np.uint8) for L in lens]
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    off[1:] = np.cumsum(lens)
    dna = np.concatenate(contigs)
    aa, so, meta = B.plast_translate6(torch.from_numpy(dna).cuda(), torch.from_numpy(off).cuda())
    w_aa, w_so, w_meta = oracle.translate6(dna, off)
    assert np.array_equal(aa.cpu().numpy(), w_aa)
    assert np.array_equal(so.cpu().numpy(), w_so)
    assert np.array_equal(meta.cpu().numpy(), w_meta)


def test_tplastn_parity_small(B):
    b1, dna = synth.tplastn_workload(seed=5, scale=0.01)
    aa, so, _ = B.plast_translate6(torch.from_numpy(dna.codes).cuda(), torch.from_numpy(dna.seq_off).cuda())
    w_aa, w_so, _ = oracle.translate6(dna.codes, dna.seq_off)
    assert np.array_equal(aa.cpu().numpy(), w_aa)
    g1, o1 = both(B, b1.codes, b1.seq_off)
    g2 = B.plast_index_bank(aa, so)
    o2 = oracle.make_bank(w_aa, w_so)
    want = oracle.ungapped(o1, o2, threads=8)
    got = B.hits_numpy(B.plast_ungapped(g1, g2))
    assert len(want) > 0
    assert same(got, want)
    recs, _ = B.plast_search_ex(g1, g2)
    w_recs = oracle.small_gapped(o1, o2, want)
    assert same(B.gapped_numpy(recs), w_recs)
    # stage 3.2 through the translated frames (extensions cross stop codons)
    al, ext = B.plast_full_gapped(g1, g2, recs)
    w_al, w_ext = oracle.full_gapped(o1, o2, w_recs, threads=8, return_extended=True)
    assert ext == w_ext and len(w_al) > 0
    assert same(B.alignments_numpy(al), w_al)


def test_errors(B):
    c, o = bank_from(["AQAAW"])
    bad = c.copy()
    bad[2] = 22
    d = B.DeviceBank.from_host(bad, o)
    with pytest.raises(B.PlastError) as e:
        B.plast_index_bank(d.codes, d.seq_off)
    assert e.value.code == B.PLAST_E_INVALID
    d = B.DeviceBank.from_host(c, np.array([0, 3, 2], dtype=np.int64))
    with pytest.raises(B.PlastError) as e:
        B.plast_index_bank(d.codes, d.seq_off)
    assert e.value.code == B.PLAST_E_INVALID
    g = gpu_bank(B, c, o)
    with pytest.raises(B.PlastError) as e:
        B.plast_ungapped(g, g, B.plast_default_params(nl=10))
    assert e.value.code == B.PLAST_E_INVALID
    # capacity: the call reports the needed count and writes nothing
    h = B.plast_ungapped(g, g, B.plast_default_params(s1=-100))
    assert h.shape[0] == 2
    with pytest.raises(B.PlastError) as e:
        B.plast_ungapped(g, g, B.plast_default_params(s1=-100), cap=1)
    assert e.value.code == B.PLAST_E_CAPACITY and e.value.needed == 2
    # small gapped on a hit outside the bank
    hit = B.hits_numpy(h)[:1].copy()
    hit["pos2"] = 99
    with pytest.raises(B.PlastError) as e:
        B.plast_small_gapped(g, g, B.hits_from_numpy(hit))
    assert e.value.code == B.PLAST_E_INVALID
    dna = torch.tensor([0, 1, 4], dtype=torch.uint8, device="cuda")
    with pytest.raises(B.PlastError) as e:
        B.plast_translate6(dna, torch.tensor([0, 3], dtype=torch.int64, device="cuda"))
    assert e.value.code == B.PLAST_E_INVALID
    # a bank whose padded length reaches 2^31 is refused before any kernel
    # reads its codes (the offsets alone are checked on the host)
    big = torch.tensor([0, 2 ** 31 - 100], dtype=torch.int64, device="cuda")
    with pytest.raises(B.PlastError) as e:
        B.plast_index_bank(torch.zeros(16, dtype=torch.int8, device="cuda"), big)
    assert e.value.code == B.PLAST_E_INVALID


def test_allocation_failure_injection(B, plain):
    # host-side fault injection: allocations above the limit fail as out of
    # memory; every call reports PLAST_E_OOM, frees what it took, and the
    # library works again once the limit is lifted
    g1, o1, g2, o2 = plain
    want, n_want = B.plast_search_ex(g1, g2)
    b1, _ = synth.workload("plastp_plain", seed=1)
    d1 = B.DeviceBank.from_host(b1.codes, b1.seq_off)
    try:
        B.plast_set_alloc_limit(4096)
        for call in (lambda: B.plast_search(g1, g2), lambda: B.plast_ungapped(g1, g2),
                     lambda: B.plast_index_bank(d1.codes, d1.seq_off),
                     lambda: B.Plan(g1, g2, max_hits=10 ** 6, max_records=10 ** 5)):
            with pytest.raises(B.PlastError) as e:
                call()
            assert e.value.code == B.PLAST_E_OOM
    finally:
        B.plast_set_alloc_limit(0)
    got, n_got = B.plast_search_ex(g1, g2)
    assert n_got == n_want and torch.equal(got, want)
    g3 = B.plast_index_bank(d1.codes, d1.seq_off)
    check_index(B, g3, o1)


def test_bank_built_on_another_stream(B):
    # the index call returns while its last kernel may still run on its
    # stream; a search on another stream must wait for it, and a free right
    # after the build must too
    b1, b2 = synth.workload("plastp_plain", seed=14, scale=0.3)
    o1, o2 = oracle.make_bank(b1.codes, b1.seq_off), oracle.make_bank(b2.codes, b2.seq_off)
    want = oracle.small_gapped(o1, o2, oracle.ungapped(o1, o2, threads=8))
    side = torch.cuda.Stream()
    d1 = B.DeviceBank.from_host(b1.codes, b1.seq_off)
    d2 = B.DeviceBank.from_host(b2.codes, b2.seq_off)
    torch.cuda.synchronize()
    for _ in range(3):
        g1 = B.plast_index_bank(d1.codes, d1.seq_off, stream=side)
        g2 = B.plast_index_bank(d2.codes, d2.seq_off, stream=side)
        recs, _ = B.plast_search_ex(g1, g2)  # current stream
        assert same(B.gapped_numpy(recs), want)
        g3 = B.plast_index_bank(d2.codes, d2.seq_off, stream=side)
        g3.free()


def test_s0_filter(B, plain):
    # Section 4.2's lossy filter: hits and records equal the oracle's
    # filter-then-extend, at the calibrated S0 and at a harsher one
    g1, o1, g2, o2 = plain
    full = oracle.ungapped(o1, o2, threads=8)
    for s0 in (B.PLAST_FILTER_S0, 70):
        want_h = oracle.ungapped(o1, o2, oracle.Params(s0=s0), threads=8)
        assert 100 < len(want_h) < len(full)
        assert same(B.hits_numpy(B.plast_ungapped_ex(g1, g2, s0=s0)), want_h)
        recs, n_ung = B.plast_search_ex(g1, g2, s0=s0)
        assert n_ung == len(want_h)
        assert same(B.gapped_numpy(recs), oracle.small_gapped(o1, o2, want_h))
        keys = np.arange(0, B.NKEYS, 7, dtype=np.int32)
        want_k = oracle.ungapped(o1, o2, oracle.Params(s0=s0), keys=keys, threads=8)
        assert same(B.hits_numpy(B.plast_ungapped_ex(g1, g2, s0=s0, keys=keys)), want_k)
    # a filter at or below S1 removes nothing (U <= F)
    assert same(B.hits_numpy(B.plast_ungapped_ex(g1, g2, s0=38)), full)
    for bad in (-1, 30001):
        with pytest.raises(B.PlastError):
            B.plast_ungapped_ex(g1, g2, s0=bad)
        with pytest.raises(B.PlastError):
            B.plast_search_ex(g1, g2, s0=bad)


def test_plastx_both_translated(B):
    # PLAST-X proper: two nucleotide banks, each translated in six frames
    q, subj = synth.plastx_workload(seed=16, scale=0.02)
    got, want = [], []
    for dna in (q, subj):
        aa, so, _ = B.plast_translate6(torch.from_numpy(dna.codes).cuda(), torch.from_numpy(dna.seq_off).cuda())
        w_aa, w_so, _ = oracle.translate6(dna.codes, dna.seq_off)
        assert np.array_equal(aa.cpu().numpy(), w_aa) and np.array_equal(so.cpu().numpy(), w_so)
        got.append(B.plast_index_bank(aa, so))
        want.append(oracle.make_bank(w_aa, w_so))
    want_h = oracle.ungapped(want[0], want[1], threads=8)
    assert len(want_h) > 1000
    assert same(B.hits_numpy(B.plast_ungapped(got[0], got[1])), want_h)
    recs, n_ung = B.plast_search_ex(got[0], got[1])
    assert n_ung == len(want_h)
    w_recs = oracle.small_gapped(want[0], want[1], want_h)
    assert same(B.gapped_numpy(recs), w_recs)
    # stage 3.2 on the translated frames (extensions run through stop codons
    # on both sides)
    al, ext = B.plast_full_gapped(got[0], got[1], recs)
    w_al, w_ext = oracle.full_gapped(want[0], want[1], w_recs, threads=8, return_extended=True)
    assert ext == w_ext and len(w_al) > 0
    assert same(B.alignments_numpy(al), w_al)


def test_plastx_translated_queries(B):
    # PLAST-X: a nucleotide query bank translated in six frames against a
    # protein bank (the queries as bank 1)
    b_prot, dna = synth.tplastn_workload(seed=15, scale=0.004)
    aa, so, _ = B.plast_translate6(torch.from_numpy(dna.codes).cuda(), torch.from_numpy(dna.seq_off).cuda())
    w_aa, w_so, _ = oracle.translate6(dna.codes, dna.seq_off)
    assert np.array_equal(aa.cpu().numpy(), w_aa) and np.array_equal(so.cpu().numpy(), w_so)
    gq = B.plast_index_bank(aa, so)
    oq = oracle.make_bank(w_aa, w_so)
    gp, op = both(B, b_prot.codes, b_prot.seq_off)
    want_h = oracle.ungapped(oq, op, threads=8)
    assert len(want_h) > 0
    assert same(B.hits_numpy(B.plast_ungapped(gq, gp)), want_h)
    recs, n_ung = B.plast_search_ex(gq, gp)
    assert n_ung == len(want_h)
    assert same(B.gapped_numpy(recs), oracle.small_gapped(oq, op, want_h))
