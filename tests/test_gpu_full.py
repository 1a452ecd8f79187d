"""Stage 3.2 on the GPU (plast_full_gapped) against the oracle's statement
of it (oracle.full_gapped): the full gapped extension with the drop-off X,
the trace-back fields and the redundant-alignment lists, byte for byte.

* the 200 x 2,000 workload whole, at the default drop-off and at others,
  with other gap costs, and with the records given in a shuffled order;
* sampled keys of the 10,000 x 100,000 workload (the records of those keys,
  from plast_search_ex, extended on both sides);
* error paths: bad records, bad drop-off, a capacity too small, and a row
  wider than the kernel's row buffer (reported, and the library still
  answers the next call).
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
    return binding


def banks(B, b1, b2):
    d1 = B.DeviceBank.from_host(b1.codes, b1.seq_off)
    d2 = B.DeviceBank.from_host(b2.codes, b2.seq_off)
    return (B.plast_index_bank(d1.codes, d1.seq_off), B.plast_index_bank(d2.codes, d2.seq_off),
            oracle.make_bank(b1.codes, b1.seq_off), oracle.make_bank(b2.codes, b2.seq_off))


def same(got, want):
    return got.shape == want.shape and np.array_equal(got.view(np.uint8), want.view(np.uint8))


@pytest.fixture(scope="module")
def plain(B):
    b1, b2 = synth.workload("plastp_plain", seed=1)
    g1, g2, o1, o2 = banks(B, b1, b2)
    recs, _ = B.plast_search_ex(g1, g2)
    return g1, g2, o1, o2, recs


def test_full_gapped_plain_whole(B, plain):
    g1, g2, o1, o2, recs = plain
    r = B.gapped_numpy(recs)
    assert len(r) > 1000
    want, ext_w = oracle.full_gapped(o1, o2, r, threads=8, return_extended=True)
    got, ext = B.plast_full_gapped(g1, g2, recs)
    assert ext == ext_w and 0 < ext < len(r)  # planted homologs give redundant hits
    assert same(B.alignments_numpy(got), want)
    # every record extended or skipped, and s3 only filters
    every, ext2 = B.plast_full_gapped(g1, g2, recs, s3=-10 ** 4)
    assert ext2 == ext and len(B.alignments_numpy(every)) == ext


@pytest.mark.parametrize("x,go,ge", [(0, 11, 1), (15, 11, 1), (100, 11, 1), (38, 5, 2), (38, 20, 3), (60, 0, 1)])
def test_full_gapped_other_parameters(B, plain, x, go, ge):
    g1, g2, o1, o2, recs = plain
    r = B.gapped_numpy(recs)
    want, ext_w = oracle.full_gapped(o1, o2, r, oracle.Params(gap_open=go, gap_extend=ge), x=x, s3=30, threads=8,
                                     return_extended=True)
    got, ext = B.plast_full_gapped(g1, g2, recs, B.plast_default_params(gap_open=go, gap_extend=ge), xdrop=x, s3=30)
    assert ext == ext_w
    assert same(B.alignments_numpy(got), want)


def test_full_gapped_input_order(B, plain):
    g1, g2, o1, o2, recs = plain
    want, _ = B.plast_full_gapped(g1, g2, recs)
    perm = torch.from_numpy(np.random.default_rng(5).permutation(recs.shape[0])).to(recs.device)
    got, _ = B.plast_full_gapped(g1, g2, recs[perm].contiguous())
    assert torch.equal(got, want)


def test_full_gapped_sampled_keys_full_size(B):
    b1, b2 = synth.workload("plastp_full", seed=1)
    g1, g2, o1, o2 = banks(B, b1, b2)
    pp = np.diff(o1.idx.key_off) * np.diff(o2.idx.key_off)
    rng = np.random.default_rng(41)
    keys = np.sort(rng.choice(np.nonzero(pp > 0)[0], size=120, replace=False)).astype(np.int32)
    recs, _ = B.plast_search_ex(g1, g2, keys=keys)
    r = B.gapped_numpy(recs)
    assert len(r) > 5000
    want, ext_w = oracle.full_gapped(o1, o2, r, threads=16, return_extended=True)
    got, ext = B.plast_full_gapped(g1, g2, recs)
    assert ext == ext_w
    assert same(B.alignments_numpy(got), want)


def test_full_gapped_errors(B, plain):
    g1, g2, o1, o2, recs = plain
    for bad in (-1, 30001):
        with pytest.raises(B.PlastError) as e:
            B.plast_full_gapped(g1, g2, recs, xdrop=bad)
        assert e.value.code == B.PLAST_E_INVALID
    r = B.gapped_numpy(recs[:10]).copy()
    r["pos1"][3] = 10 ** 6  # beyond its sequence
    t = torch.from_numpy(r.view(np.uint8).reshape(-1, B.GAPPED_BYTES).copy()).cuda()
    with pytest.raises(B.PlastError) as e:
        B.plast_full_gapped(g1, g2, t)
    assert e.value.code == B.PLAST_E_INVALID
    with pytest.raises(B.PlastError) as e:
        B.plast_full_gapped(g1, g2, recs, cap=1)
    assert e.value.code == B.PLAST_E_CAPACITY and e.value.needed > 1
    empty, ext = B.plast_full_gapped(g1, g2, recs[:0])
    assert empty.shape[0] == 0 and ext == 0


def test_full_gapped_row_wider_than_the_kernel_holds(B, plain):
    # free gaps and the largest drop-off keep every cell of a 3,000-residue
    # row alive, wider than the 1,024 columns a row buffer holds: the call
    # reports PLAST_E_CAPACITY and returns nothing partial
    rng = np.random.default_rng(3)
    codes = rng.integers(0, 20, size=3000).astype(np.int8)
    off = np.array([0, 3000], dtype=np.int64)
    d = B.DeviceBank.from_host(codes, off)
    g = B.plast_index_bank(d.codes, d.seq_off)
    r = np.zeros(1, dtype=B.GAPPED_DTYPE)
    r["pos1"] = r["pos2"] = 100
    t = torch.from_numpy(r.view(np.uint8).reshape(-1, B.GAPPED_BYTES).copy()).cuda()
    with pytest.raises(B.PlastError) as e:
        B.plast_full_gapped(g, g, t, B.plast_default_params(gap_open=0, gap_extend=0), xdrop=30000)
    assert e.value.code == B.PLAST_E_CAPACITY
    assert B.plast_full_gapped_cells() == 0
    # the same record at the default costs fits, and the library recovers;
    # the anchor sits on the main diagonal of a sequence against itself, so
    # both sides run to the sequence ends: at least one cell per row
    got, ext = B.plast_full_gapped(g, g, t)
    want = oracle.full_gapped(oracle.make_bank(codes, off), oracle.make_bank(codes, off), r)
    assert ext == 1 and same(B.alignments_numpy(got), want)
    assert B.plast_full_gapped_cells() >= 3000
    g1, g2, o1, o2, recs = plain
    again, _ = B.plast_full_gapped(g1, g2, recs)
    assert same(B.alignments_numpy(again), oracle.full_gapped(o1, o2, B.gapped_numpy(recs), threads=8))


def test_full_gapped_largest_drop_off_and_free_gaps(B):
    # X = 30000 keeps every cell alive: the rows' int16 values, relative to
    # the drop-off line, reach X + 11, the edge of their range; free gaps
    # (go = ge = 0) make E and F tie with the diagonal everywhere and keep
    # whole rows alive too.  Sequences of at most 400 residues keep a side
    # within the kernel's working space (longer ones get PLAST_E_CAPACITY);
    # the records are anchors drawn at random (stage 3.2 takes any record),
    # some on planted homologs, several per pair of sequences
    rng = np.random.default_rng(9)
    src = synth.random_protein_bank(rng, 12)
    seqs = [src.seq(i)[:400] for i in range(12)]
    codes = np.concatenate(seqs).astype(np.int8)
    off = np.zeros(13, dtype=np.int64)
    np.cumsum([len(q) for q in seqs], out=off[1:])
    hom = [synth.mutate(rng, q, 0.7)[:400] for q in seqs[:6]] + [src.seq(i)[:400] for i in range(6, 12)]
    codes2 = np.concatenate(hom).astype(np.int8)
    off2 = np.zeros(13, dtype=np.int64)
    np.cumsum([len(q) for q in hom], out=off2[1:])
    g1, g2, o1, o2 = banks(B, synth.SynthBank(codes, off), synth.SynthBank(codes2, off2))
    r = np.zeros(60, dtype=B.GAPPED_DTYPE)
    r["seq1"] = rng.integers(0, 12, size=60)
    r["seq2"] = np.where(rng.random(60) < 0.6, r["seq1"], rng.integers(0, 12, size=60))
    r["pos1"] = [rng.integers(0, off[s + 1] - off[s]) for s in r["seq1"]]
    r["pos2"] = [rng.integers(0, off2[s + 1] - off2[s]) for s in r["seq2"]]
    r["score"] = rng.integers(40, 200, size=60)
    t = torch.from_numpy(r.view(np.uint8).reshape(-1, B.GAPPED_BYTES).copy()).cuda()
    for x, go, ge in ((30000, 11, 1), (5000, 11, 1), (20, 0, 0), (30000, 0, 0)):
        want, ext_w = oracle.full_gapped(o1, o2, r, oracle.Params(gap_open=go, gap_extend=ge), x=x, s3=-10 ** 6,
                                         return_extended=True)
        got, ext = B.plast_full_gapped(g1, g2, t, B.plast_default_params(gap_open=go, gap_extend=ge), xdrop=x,
                                       s3=-10 ** 6)
        assert ext == ext_w and same(B.alignments_numpy(got), want), (x, go, ge)
