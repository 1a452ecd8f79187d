"""The tabular form of the stage-4 records (BLAST's -m 8 column order,
Section 3.3.5): a record written out by hand, and the oracle's alignments of
a sequence against itself, whose lines are fixed by the identity closed
form (every residue aligned with itself: 100 % identity, no mismatch, no
gap, coordinates 1 .. length)."""
import numpy as np

import oracle
from paper_0804_3643_gb300 import binding as B
from paper_0804_3643_gb300 import synth


def test_hand_written_record():
    r = np.zeros(1, dtype=B.ALIGN_DTYPE)
    r["seq1"], r["seq2"], r["pos1"], r["pos2"] = 3, 7, 10, 12
    r["score"] = 85
    r["q_start"], r["q_end"], r["s_start"], r["s_end"] = 4, 44, 5, 46
    r["length"], r["identities"], r["mismatches"], r["gap_opens"] = 41, 30, 10, 1
    (line,) = B.alignments_tabular(r, names1={3: "q3"}, names2={7: "s7"})
    assert line.split("\t") == ["q3", "s7", "73.17", "41", "10", "1", "5", "44", "6", "46", "85"]


def test_self_alignment_lines():
    rng = np.random.default_rng(5)
    bank = synth.random_protein_bank(rng, 3)
    o = oracle.make_bank(bank.codes, bank.seq_off)
    r = np.zeros(3, dtype=B.GAPPED_DTYPE)
    r["seq1"] = r["seq2"] = np.arange(3)
    r["pos1"] = r["pos2"] = [5, 9, 2]
    al = oracle.full_gapped(o, o, r, x=30000, s3=0)
    lines = B.alignments_tabular(al)
    assert len(lines) == 3
    for s, line in enumerate(lines):
        n = int(bank.seq_off[s + 1] - bank.seq_off[s])
        f = line.split("\t")
        assert f[:10] == [str(s), str(s), "100.00", str(n), "0", "0", "1", str(n), "1", str(n)]
