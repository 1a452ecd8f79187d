"""Sanity metric for the whole method on the small workload (no GPU): every
bank-2 protein planted as a mutated copy (identity 40-90 %, indels) of a
bank-1 protein comes out of stages 1-3.1 as at least one record pairing the
two, near their common diagonal (the recall criterion the paper's
sensitivity comparison builds on, Annex 2).  The GPU path's records equal
the oracle's (tests/test_gpu_parity.py), so the same holds there."""
import numpy as np

import oracle
from paper_0804_3643_gb300 import synth


def test_planted_homologs_recalled():
    b1, b2 = synth.workload("plastp_plain", seed=1)
    o1, o2 = oracle.make_bank(b1.codes, b1.seq_off), oracle.make_bank(b2.codes, b2.seq_off)
    rec = oracle.small_gapped(o1, o2, oracle.ungapped(o1, o2, threads=16))
    planted = b2.planted
    assert len(planted["bank2_index"]) == 200
    found = 0
    for i, j in zip(planted["bank2_index"], planted["bank1_source"]):
        on = (rec["seq1"] == j) & (rec["seq2"] == i)
        # a mutated full-length copy: the record lies near the main diagonal
        # (indels of at most 10 residues at rate 0.02 shift it a little)
        if on.any() and np.abs(rec["pos2"][on] - rec["pos1"][on]).min() <= 30:
            found += 1
    assert found >= 0.95 * len(planted["bank2_index"]), found
