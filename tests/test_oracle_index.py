"""Pins of the oracle's stage 0 (Section 3.3.1): the CSR index equals a
brute-force enumeration of every overlapping word inside each sequence."""
import numpy as np

import oracle
from conftest import bank_from, enc, golden


def brute_index(codes, seq_off):
    lists = {}
    for s in range(len(seq_off) - 1):
        for p in range(int(seq_off[s]), int(seq_off[s + 1]) - 3):
            k = oracle.seed_key(codes[p:p + 4])
            if k >= 0:
                lists.setdefault(k, []).append(p)
    return lists


def check_index(codes, seq_off):
    idx = oracle.index(codes, seq_off)
    want = brute_index(codes, seq_off)
    assert idx.key_off[0] == 0 and (np.diff(idx.key_off) >= 0).all()
    assert idx.key_off[-1] == sum(len(v) for v in want.values()) == len(idx.pos)
    for k in range(oracle.NKEYS):
        got = idx.pos[idx.key_off[k]:idx.key_off[k + 1]].tolist()
        assert got == want.get(k, []), k


def test_overlapping_words_of_printed_example():
    g = golden("word_split.txt")
    seq = g["sequence"]
    codes, off = bank_from([seq])
    idx = oracle.index(codes, off)
    # every start p with p + 3 < len is a word: overlapping, one per letter
    assert len(idx.pos) == len(seq) - 3
    assert sorted(idx.pos.tolist()) == list(range(len(seq) - 3))
    # the printed W = 3 words are the prefixes of consecutive words
    w3 = g["first words"].split()
    for p, w in enumerate(w3):
        assert seq[p:p + int(g["w"])] == w


def test_index_matches_brute_force_random(rng):
    for trial in range(5):
        n = int(rng.integers(1, 8))
        seqs = [rng.integers(0, 20, int(rng.integers(1, 60))).astype(np.int8) for _ in range(n)]
        check_index(*bank_from(seqs))


def test_index_low_complexity_and_stops(rng):
    # repeated words give long lists; stops are never inside an indexed word
    seqs = ["AAAAAAAAAAAAAAAAAAAA", "AQAAPAAASAAA*AAAA", "W", "", "MKV*", "AQA"]
    codes, off = bank_from(seqs)
    check_index(codes, off)
    idx = oracle.index(codes, off)
    for p in idx.pos:
        assert 20 not in codes[p:p + 4].tolist()
    # no word crosses a sequence boundary
    ends = set(off[1:].tolist())
    for p in idx.pos:
        assert not any(p < e < p + 4 for e in ends)


def test_index_empty_bank():
    codes, off = bank_from([])
    idx = oracle.index(codes, off)
    assert len(idx.pos) == 0 and idx.key_off[-1] == 0
    codes, off = bank_from(["", "AB"[:0]])
    assert len(oracle.index(codes, off).pos) == 0
