"""Stage-2 tile shapes: wide-only, narrow-only (16, 8, 4, 2 rows) and by-cost work lists give the
oracle's hits and records bit for bit (shapes change the schedule, never the
results), on the plain workload, a small query bank against a large bank
(ragged narrow tiles), a two-protein query whose wide tiles are cut along
their bank-2 lists, the low-complexity mix and the every-pair-passes case
(per-warp buffer overflow in narrow tiles); the calibration returns usable
costs."""
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
    yield binding
    binding.plast_set_tile_shape(0)


def both(B, codes, seq_off):
    d = B.DeviceBank.from_host(codes, seq_off)
    return B.plast_index_bank(d.codes, d.seq_off), oracle.make_bank(codes, seq_off)


def same(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint8), b.view(np.uint8))


def each_shape(B, f):
    out = []
    try:
        for shape in (1, 2, 3, 4, 5, 0):
            B.plast_set_tile_shape(shape)
            out.append(f())
    finally:
        B.plast_set_tile_shape(0)
    return out


def test_shapes_plain(B):
    b1, b2 = synth.workload("plastp_plain", seed=7, scale=0.5)
    g1, o1 = both(B, b1.codes, b1.seq_off)
    g2, o2 = both(B, b2.codes, b2.seq_off)
    want_h = oracle.ungapped(o1, o2, threads=16)
    want = oracle.small_gapped(o1, o2, want_h)
    assert len(want_h) > 500
    for h in each_shape(B, lambda: B.hits_numpy(B.plast_ungapped(g1, g2))):
        assert same(h, want_h)
    for r, n in each_shape(B, lambda: B.plast_search_ex(g1, g2)):
        assert n == len(want_h) and same(B.gapped_numpy(r), want)


def test_small_query_large_bank(B):
    rng = np.random.default_rng(11)
    bank = synth.protein_bank(rng, 6000)
    q = synth.random_protein_bank(np.random.default_rng(12), 23)
    # plus mutated copies of bank proteins, so that hits exist
    seqs = [q.seq(i) for i in range(q.n_seqs)]
    seqs += [synth.mutate(rng, bank.seq(int(rng.integers(0, bank.n_seqs))), 0.6) for _ in range(9)]
    c, o = bank_from(seqs)
    gq, oq = both(B, c, o)
    gb, ob = both(B, bank.codes, bank.seq_off)
    tiles = B.plast_stage2_tiles(oq.idx.key_off, ob.idx.key_off)
    assert (tiles[:, 3] >= 1).mean() > 0.9  # by cost, almost all narrow
    assert len(set(tiles[:, 3].tolist())) >= 2
    assert ((tiles[:, 2] % 8) != 0).any()    # ragged narrow tiles
    want_h = oracle.ungapped(oq, ob, threads=16)
    want = oracle.small_gapped(oq, ob, want_h)
    assert len(want) > 20
    for h in each_shape(B, lambda: B.hits_numpy(B.plast_ungapped(gq, gb))):
        assert same(h, want_h)
    for r, n in each_shape(B, lambda: B.plast_search_ex(gq, gb)):
        assert n == len(want_h) and same(B.gapped_numpy(r), want)
    # the query as bank 2: wide rows from the large bank, few windows per key
    want_sw = oracle.ungapped(ob, oq, threads=16)
    for h in each_shape(B, lambda: B.hits_numpy(B.plast_ungapped(gb, gq))):
        assert same(h, want_sw)


def test_wide_tiles_cut(B):
    # a two-protein query against a large bank: a few hundred keys, fewer
    # tiles than CTAs; with the shape forced wide the costliest wide tiles
    # are cut along their bank-2 lists into pieces of whole 128-window passes
    rng = np.random.default_rng(21)
    bank = synth.protein_bank(rng, 12000)
    c, o = bank_from([synth.mutate(rng, bank.seq(int(rng.integers(0, bank.n_seqs))), 0.6) for _ in range(2)])
    gq, oq = both(B, c, o)
    gb, ob = both(B, bank.codes, bank.seq_off)
    n_sms = torch.cuda.get_device_properties(0).multi_processor_count
    try:
        B.plast_set_tile_shape(1)
        whole = B.plast_stage2_tiles(oq.idx.key_off, ob.idx.key_off)
        cut = B.plast_stage2_tiles(oq.idx.key_off, ob.idx.key_off, n_sms=n_sms)
    finally:
        B.plast_set_tile_shape(0)
    assert (whole[:, 3] == 0).all() and (cut[:, 3] == 0).all() and len(cut) > len(whole)
    assert ((cut[:, 5] - cut[:, 4]) % 128 != 0).any()   # ragged last pieces
    want_h = oracle.ungapped(oq, ob, threads=16)
    want = oracle.small_gapped(oq, ob, want_h)
    assert len(want_h) > 100
    for h in each_shape(B, lambda: B.hits_numpy(B.plast_ungapped(gq, gb))):
        assert same(h, want_h)
    for r, n in each_shape(B, lambda: B.plast_search_ex(gq, gb)):
        assert n == len(want_h) and same(B.gapped_numpy(r), want)


def test_shapes_low_complexity(B):
    b1, b2 = synth.workload("batching_stress", seed=9, scale=0.003)
    g1, o1 = both(B, b1.codes, b1.seq_off)
    g2, o2 = both(B, b2.codes, b2.seq_off)
    want = oracle.ungapped(o1, o2, threads=16)
    for h in each_shape(B, lambda: B.hits_numpy(B.plast_ungapped(g1, g2))):
        assert same(h, want)


def test_narrow_every_pair_passes(B):
    rng = np.random.default_rng(13)
    seqs = [rng.integers(0, 4, int(rng.integers(20, 120))).astype(np.int8) for _ in range(25)]
    c, o = bank_from(seqs)
    g, ob = both(B, c, o)
    prm = oracle.Params(s1=0)
    want = oracle.ungapped(ob, ob, prm)
    for h in each_shape(B, lambda: B.hits_numpy(B.plast_ungapped(g, g, B.plast_default_params(s1=0)))):
        assert same(h, want)


def test_autotune(B):
    saved = B.plast_get_tile_costs()
    try:
        c = B.plast_autotune()
        assert c["wide_slot"] > 0 and c["narrow_slot"] > 0
        assert c["wide_tile"] >= 0 and c["narrow_tile"] >= 0
        # a row slot of either shape costs 48 cells: between 0.01 and 10 SM-ns
        assert 0.01 < c["wide_slot"] < 10 and 0.01 < c["narrow_slot"] < 10
        assert 0.01 < c["narrow16_slot"] < 10 and c["narrow16_tile"] >= 0
        assert B.plast_get_tile_costs() == c
    finally:
        B.plast_set_tile_costs(saved)


def test_wide_variants_parity(B):
    # every wide-kernel variant (int16 cells 0, 12, 14, 16; bank-2 windows
    # fetched one or two passes ahead) gives the oracle's hits, with full
    # tiles, a ragged last tile and rows of sentinels; bank 2 large enough
    # that keys span several passes of 96 windows
    b1, b2 = synth.workload("plastp_plain", seed=8, scale=0.5, n2=8000)
    g1, o1 = both(B, b1.codes, b1.seq_off)
    g2, o2 = both(B, b2.codes, b2.seq_off)
    want = oracle.ungapped(o1, o2, threads=16)
    prm = oracle.Params(s1=20)
    want20 = oracle.ungapped(o1, o2, prm, threads=16)
    saved = B.plast_get_tile_costs()
    try:
        B.plast_set_tile_shape(1)
        for n16 in (0, 12, 14, 16):
            for depth in (1, 2):
                B.plast_set_tile_costs(dict(saved, wide_int16_cells=n16, wide_stage_depth=depth))
                assert same(B.hits_numpy(B.plast_ungapped(g1, g2)), want)
                assert same(B.hits_numpy(B.plast_ungapped(g1, g2, B.plast_default_params(s1=20))), want20)
    finally:
        B.plast_set_tile_shape(0)
        B.plast_set_tile_costs(saved)
