"""Pins of the oracle's stage 3.2 (full gapped extension with the row-wise
drop-off X, Sections 2.3.3 and 3.3.4), its trace-back to BLAST's tabular
fields (Section 3.3.5) and the redundant-alignment lists (Section 3.3.4):
closed forms worked by hand, Smith-Waterman as a bound and (without a
drop-off) as the maximum over anchors, the alignment rescored from its own
columns, the redundancy check worked by hand and independence of the input
order."""
import numpy as np

import oracle
from conftest import enc

BIG_X = 10 ** 5  # a drop-off no score can reach: the plain anchored extension
B62 = oracle.blosum62()


def diag_sum(s: str) -> int:
    return sum(int(B62[c, c]) for c in enc(s))


def test_identity_closed_form():
    # x against itself through any anchor: every column scores its diagonal
    # entry (> 0), so the whole sequence aligns without gaps
    x = "MKTAYIAKQRQISFVKSHFSRQLEERLGLIEVQ"
    for p in (0, 7, len(x) - 1):
        al, segs = oracle.full_gapped_one(enc(x), p, enc(x), p)
        assert al["score"] == diag_sum(x)
        assert (al["q_start"], al["q_end"], al["s_start"], al["s_end"]) == (0, len(x), 0, len(x))
        assert al["length"] == al["identities"] == len(x) and al["mismatches"] == al["gap_opens"] == 0
        assert segs == [(0, 0, len(x) - 1)]


def test_drop_off_stop_worked_by_hand():
    # W/W scores 11, P/W scores -4.  With a gap opening of 100 only the
    # diagonal lives: 5 x 11 = 55, four mismatches take it down 16 to 39,
    # five more matches bring it to 94.  A drop-off of 15 kills the row where
    # the dip reaches 16 (39 < 55 - 15) and the side ends at 55; one of 16
    # lets it through.
    x, y = enc("WWWWW" + "PPPP" + "WWWWW"), enc("WWWWW" + "WWWW" + "WWWWW")
    assert oracle.score(enc("P")[0], enc("W")[0]) == -4 and oracle.score(enc("W")[0], enc("W")[0]) == 11
    assert oracle.xdrop_side(x, y, go=100, ge=1, x=15)[:3] == (55, 5, 5)
    assert oracle.xdrop_side(x, y, go=100, ge=1, x=16)[:3] == (94, 14, 14)
    assert oracle.xdrop_side(x, y, go=100, ge=1, x=16)[3] == "M" * 14


def test_single_gap_worked_by_hand():
    # ten W against five W, a G, five W: the G is skipped by one gap of
    # length 1 (cost 11 + 1): 10 x 11 - 12 = 98, better than the ungapped
    # 5 x 11 - 2 + 4 x 11 = 97
    x, y = enc("W" * 10), enc("WWWWWGWWWWW")
    sc, ei, ej, path = oracle.xdrop_side(x, y)
    assert (sc, ei, ej) == (98, 10, 11)
    assert path.count("D") == 1 and path.count("M") == 10 and path.count("I") == 0
    al, segs = oracle.full_gapped_one(x, 0, y, 0)
    assert al["score"] == 98 and al["gap_opens"] == 1 and al["length"] == 11
    assert al["identities"] == 10 and al["mismatches"] == 0
    # two gap-free runs on the diagonals 0 and -1
    assert segs == [(0, 0, 4), (-1, 5, 9)]


def rescore(x, y, al, segs, go=11, ge=1):
    """Score of an alignment from its own columns: the residue pairs of its
    gap-free segments, minus go + k * ge per gap run."""
    m = sum(int(B62[x[k], y[k - d]]) for d, a, b in segs for k in range(a, b + 1))
    pairs = sum(b - a + 1 for d, a, b in segs)
    gap_cols = int(al["length"]) - pairs
    return m - go * int(al["gap_opens"]) - ge * gap_cols, pairs


def test_alignments_rescore_to_their_score(rng):
    # random homologous pairs (mutations and indels): the fields reported by
    # the trace-back add up to the dynamic programme's score, the path runs
    # through the anchor and its extents match the coordinates
    from paper_0804_3643_gb300 import synth

    b1, b2 = synth.workload("plastp_plain", seed=9, scale=0.05)
    o1, o2 = oracle.make_bank(b1.codes, b1.seq_off), oracle.make_bank(b2.codes, b2.seq_off)
    recs = oracle.small_gapped(o1, o2, oracle.ungapped(o1, o2))
    assert len(recs) > 30
    for r in recs[rng.choice(len(recs), size=min(60, len(recs)), replace=False)]:
        x = o1.codes[o1.seq_off[r["seq1"]]:o1.seq_off[r["seq1"] + 1]]
        y = o2.codes[o2.seq_off[r["seq2"]]:o2.seq_off[r["seq2"] + 1]]
        al, segs = oracle.full_gapped_one(x, int(r["pos1"]), y, int(r["pos2"]))
        sc, pairs = rescore(x, y, al, segs)
        assert sc == al["score"]
        assert pairs == al["identities"] + al["mismatches"]
        assert al["identities"] == sum(int(x[k] == y[k - d]) for d, a, b in segs for k in range(a, b + 1))
        assert al["q_start"] <= r["pos1"] <= al["q_end"] and al["s_start"] <= r["pos2"] <= al["s_end"]
        gaps = int(al["length"]) - pairs
        assert (al["q_end"] - al["q_start"]) + (al["s_end"] - al["s_start"]) == 2 * pairs + gaps
        assert al["score"] <= oracle.smith_waterman(x, y)


def test_smith_waterman_equals_max_over_anchors_without_drop_off(rng):
    # with no drop-off the anchored extension is the best alignment through
    # the anchor; its maximum over all anchors is the local optimum
    for _ in range(25):
        x = rng.integers(0, 20, int(rng.integers(3, 14))).astype(np.int8)
        y = x.copy() if rng.random() < 0.5 else rng.integers(0, 20, int(rng.integers(3, 14))).astype(np.int8)
        if rng.random() < 0.5 and len(y) > 3:
            y = np.delete(y, int(rng.integers(1, len(y) - 1)))
        best = max(oracle.full_gapped_one(x, p1, y, p2, x=BIG_X)[0]["score"]
                   for p1 in range(len(x)) for p2 in range(len(y)))
        assert best == oracle.smith_waterman(x, y)


def test_no_drop_off_is_at_least_the_small_extension(rng):
    # without a drop-off every path of the banded, LG-limited extension of
    # stage 3.1 is a path of the full one
    from paper_0804_3643_gb300 import synth

    b1, b2 = synth.workload("plastp_plain", seed=10, scale=0.05)
    o1, o2 = oracle.make_bank(b1.codes, b1.seq_off), oracle.make_bank(b2.codes, b2.seq_off)
    recs = oracle.small_gapped(o1, o2, oracle.ungapped(o1, o2), oracle.Params(s2=-10 ** 4))
    for r in recs[rng.choice(len(recs), size=min(40, len(recs)), replace=False)]:
        x = o1.codes[o1.seq_off[r["seq1"]]:o1.seq_off[r["seq1"] + 1]]
        y = o2.codes[o2.seq_off[r["seq2"]]:o2.seq_off[r["seq2"] + 1]]
        al, _ = oracle.full_gapped_one(x, int(r["pos1"]), y, int(r["pos2"]), x=BIG_X)
        assert al["score"] >= r["score"]


def gapped_records(rows):
    a = np.zeros(len(rows), dtype=oracle.GAPPED_DTYPE)
    for k, (s1, p1, s2, p2, sc) in enumerate(rows):
        a[k]["seq1"], a[k]["pos1"], a[k]["seq2"], a[k]["pos2"], a[k]["score"] = s1, p1, s2, p2, sc
    return a


def bank(*seqs):
    codes = np.concatenate([enc(s) for s in seqs])
    off = np.concatenate([[0], np.cumsum([len(s) for s in seqs])]).astype(np.int64)
    return oracle.make_bank(codes, off)


def test_redundancy_worked_by_hand():
    # sequence 0 of both banks: the same 40 residues, so the alignment
    # through any anchor on diagonal 0 covers the whole diagonal.  Taken by
    # decreasing score, the hit at 20 (score 90) is extended first; the
    # hits at 0 and 33 lie on its segment (diagonal 0, residues 0..39) and
    # are skipped.  The hit at (12, 10) lies on diagonal 2: not covered,
    # extended.  Sequence pair (0, 1) has its own list: its hit is extended.
    s = "MKTAYIAKQRQISFVKSHFSRQLEERLGLIEVQAPILSRV"
    b1 = bank(s)
    b2 = bank(s, "GGGGGGGGGG" + s[:20])
    recs = gapped_records([(0, 0, 0, 0, 60), (0, 20, 0, 20, 90), (0, 33, 0, 33, 50), (0, 12, 0, 10, 55),
                           (0, 0, 1, 10, 80)])
    out, ext = oracle.full_gapped(b1, b2, recs, s3=-10 ** 4, return_extended=True)
    assert ext == 3
    assert [(r["seq1"], r["pos1"], r["seq2"], r["pos2"]) for r in out] == [(0, 0, 1, 10), (0, 12, 0, 10), (0, 20, 0, 20)]
    whole = out[2]
    assert whole["score"] == diag_sum(s) and whole["length"] == 40 and whole["gap_opens"] == 0
    # the same records with the high-scoring anchor removed: the hit at 0 is
    # now extended first and covers 33
    out2, ext2 = oracle.full_gapped(b1, b2, recs[[0, 2, 3, 4]], s3=-10 ** 4, return_extended=True)
    assert ext2 == 3 and [int(r["pos1"]) for r in out2] == [0, 0, 12]
    # s3 keeps only the alignments that reach it (redundancy unchanged)
    out3, ext3 = oracle.full_gapped(b1, b2, recs, s3=diag_sum(s), return_extended=True)
    assert ext3 == 3 and len(out3) == 1 and out3[0]["pos1"] == 20


def test_result_does_not_depend_on_input_order(rng):
    from paper_0804_3643_gb300 import synth

    b1, b2 = synth.workload("plastp_plain", seed=12, scale=0.1)
    o1, o2 = oracle.make_bank(b1.codes, b1.seq_off), oracle.make_bank(b2.codes, b2.seq_off)
    recs = oracle.small_gapped(o1, o2, oracle.ungapped(o1, o2))
    out, ext = oracle.full_gapped(o1, o2, recs, return_extended=True)
    assert 0 < ext < len(recs) and len(out) > 0  # planted homologs give redundant hits
    for _ in range(3):
        perm = recs[rng.permutation(len(recs))]
        assert np.array_equal(oracle.full_gapped(o1, o2, perm).view(np.uint8), out.view(np.uint8))
    # threads share the pairs of sequences without changing anything
    assert np.array_equal(oracle.full_gapped(o1, o2, recs, threads=4).view(np.uint8), out.view(np.uint8))
