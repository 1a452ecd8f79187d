"""The PLAST-X workload through the oracle (no GPU): homologs planted in two
nucleotide banks, on either strand and in any frame, come out as records
between the translated sequences of their frames (contig-major, frames +1,
+2, +3, -1, -2, -3) on the diagonal where they were planted, so the
generator, the six-frame translation's numbering and positions and stages
1-3.1 agree with one another (Sections 6-7: both banks translated)."""
import numpy as np

import oracle
from paper_0804_3643_gb300 import synth


def frame_of(bank, region):
    """(translated sequence, first aa) of a planted region: frame +f starts
    at nt f - 1, frame -f at nt f - 1 of the reverse complement."""
    _, c, st, strand, n = (int(x) for x in region)
    length = int(bank.seq_off[c + 1] - bank.seq_off[c])
    a = st if not strand else length - (st + n)
    return 6 * c + 3 * strand + a % 3, a // 3


def test_planted_pairs_found():
    q, subj = synth.plastx_workload(seed=1, scale=0.05)
    qa, qo, _ = oracle.translate6(q.codes, q.seq_off)
    sa, so, _ = oracle.translate6(subj.codes, subj.seq_off)
    assert len(qa) > 10 ** 5 and len(sa) > 4 * 10 ** 6
    o1, o2 = oracle.make_bank(qa, qo), oracle.make_bank(sa, so)
    rec = oracle.small_gapped(o1, o2, oracle.ungapped(o1, o2, threads=16))
    both = found = 0
    strands = set()
    for qr in q.planted["regions"]:
        for sr in subj.planted["regions"]:
            if qr[0] != sr[0]:
                continue
            both += 1
            s1, p1 = frame_of(q, qr)
            s2, p2 = frame_of(subj, sr)
            on = (rec["seq1"] == s1) & (rec["seq2"] == s2) & (np.abs((rec["pos2"] - rec["pos1"]) - (p2 - p1)) <= 40)
            if on.any():
                found += 1
                strands.add((int(qr[3]), int(sr[3])))
    # two independent mutations of one source at 40-90 % identity each: most
    # pairs keep a seed and a window above S1
    assert both >= 8 and found >= 0.7 * both
    assert len(strands) >= 2
