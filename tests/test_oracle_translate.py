"""Pins of the oracle's six-frame translation (Section 6, TPLAST-N).

* a hand-worked contig in all six frames;
* proteins back-translated with the input generator's own codon lists are
  recovered in their frame (two independent transcriptions of the code
  agree);
* frame lengths and ordering; reverse complement twice is the identity.
"""
import numpy as np

import oracle
from conftest import AA, enc
from paper_0804_3643_gb300 import synth

NT = {"A": 0, "C": 1, "G": 2, "T": 3}


def dna(s):
    return np.array([NT[c] for c in s], dtype=np.uint8)


def frames(s):
    aa, off, meta = oracle.translate6(dna(s), [0, len(s)])
    return ["".join("*" if c == 20 else AA[c] for c in aa[off[i]:off[i + 1]]) for i in range(6)], meta


def test_hand_worked_contig():
    # ATG GCC TAA G  (10 nt)
    s = "ATGGCCTAAG"
    f, meta = frames(s)
    assert f[0] == "MA*"          # ATG GCC TAA
    # frame +2: TGG CCT AAG -> W P K
    assert f[1] == "WPK"
    # frame +3: GGC CTA -> G L
    assert f[2] == "GL"
    # reverse complement: CTTAGGCCAT
    # -1: CTT AGG CCA -> L R P ; -2: TTA GGC CAT -> L G H ; -3: TAG GCC -> * A
    assert f[3] == "LRP" and f[4] == "LGH" and f[5] == "*A"
    assert meta.tolist() == [[0, 1], [0, 2], [0, 3], [0, -1], [0, -2], [0, -3]]


def test_back_translation_round_trip():
    rng = np.random.default_rng(7)
    for _ in range(30):
        prot = rng.integers(0, 20, int(rng.integers(1, 80))).astype(np.int8)
        nt = synth.back_translate(rng, prot)
        aa, off, _ = oracle.translate6(nt, [0, len(nt)])
        assert (aa[off[0]:off[1]] == prot).all()
        rc = (3 - nt[::-1]).astype(np.uint8)
        aa2, off2, _ = oracle.translate6(rc, [0, len(rc)])
        assert (aa2[off2[3]:off2[4]] == prot).all()  # frame -1 of the reverse strand
        assert ((3 - rc[::-1]) == nt).all()


def test_frame_lengths_and_contigs():
    rng = np.random.default_rng(8)
    lens = [0, 1, 2, 3, 4, 5, 6, 7, 100, 101, 102]
    contigs = [rng.integers(0, 4, L).astype(np.uint8) for L in lens]
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    off[1:] = np.cumsum(lens)
    aa, soff, meta = oracle.translate6(np.concatenate(contigs), off)
    assert len(soff) == 6 * len(lens) + 1
    for c, L in enumerate(lens):
        for f in range(6):
            n = soff[6 * c + f + 1] - soff[6 * c + f]
            assert n == max(0, (L - (f % 3)) // 3)
            assert tuple(meta[6 * c + f]) == (c, [1, 2, 3, -1, -2, -3][f])
