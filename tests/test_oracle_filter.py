"""Pins of the oracle's Section 4.2 filter (raw score = sum of the positive
substitution scores over the ungapped window; a pair is extended only if it
reaches S0).

* hand-worked windows from published BLOSUM62 entries, with clipping;
* identity closed form: a sequence against itself sums the diagonal;
* bound: every prefix sum of the ungapped extension is at most the sum of
  the positive terms, so U <= F for every pair, and a filter with S0 <= S1
  changes nothing;
* the filtered hit set is the unfiltered one restricted to F >= S0 (the two
  gates commute), shrinking as S0 grows; the count of pairs let through
  equals a brute-force count.
"""
import numpy as np

import oracle
from conftest import AA, bank_from, enc, golden

P = oracle.Params()
DIAG = {a: int(v) for a, v in (x.split("=") for x in golden("blosum62_published.txt")["diagonal"].split())}


def test_hand_worked_windows():
    # BLOSUM62: A/A 4, W/C -2, R/K 2, D/E 2, I/V 3, G/W -2
    a, b = enc("AWRDIG"), enc("ACKEVW")
    assert oracle.filter_pair(a, 0, b, 0) == 4 + 2 + 2 + 3
    # the ungapped score of the same window: prefix sums 4, 2, 4, 6, 9, 7
    assert oracle.ungapped_pair(a, 0, b, 0)[0] == 9
    # seed at 3: left cells R/K 2, W/C -2, A/A 4; right cells D/E 2, I/V 3, G/W -2
    assert oracle.filter_pair(a, 3, b, 3) == 2 + 4 + 2 + 3
    # all-negative window: W/A -3 everywhere
    assert oracle.filter_pair(enc("WWWWWW"), 2, enc("AAAAAA"), 2) == 0
    # clipping: b ends after 2 residues right of the seed, a's extra residues
    # do not count; left side clipped by a's start
    a, b = enc("AAAAAAAA"), enc("CAAA")
    assert oracle.filter_pair(a, 0, b, 2) == 2 * 4
    assert oracle.filter_pair(a, 2, b, 1) == 3 * 4  # left: one cell, A/C 0; right: three cells A/A


def test_window_is_22_plus_26():
    a = enc("A" * 80)
    assert oracle.filter_pair(a, 30, a, 30) == 4 * 48
    assert oracle.filter_pair(a, 30, a, 5) == 4 * (26 + 5)


def test_identity_closed_form(rng):
    for _ in range(200):
        L = int(rng.integers(4, 120))
        s = rng.integers(0, 20, L).astype(np.int8)
        p = int(rng.integers(0, L - 3))
        tr, tl = min(26, L - p), min(22, p)
        f = oracle.filter_pair(s, p, s, p)
        assert f == sum(DIAG[AA[c]] for c in s[p - tl:p + tr])
        assert f == oracle.ungapped_pair(s, p, s, p)[0]
    t = enc(AA)
    assert oracle.filter_pair(t, 0, t, 0) == 116


def test_bound_u_le_f(rng):
    for _ in range(3000):
        L1, L2 = int(rng.integers(4, 70)), int(rng.integers(4, 70))
        a = rng.integers(0, 20, L1).astype(np.int8)
        b = rng.integers(0, 20, L2).astype(np.int8)
        p1, p2 = int(rng.integers(0, L1)), int(rng.integers(0, L2))
        u = oracle.ungapped_pair(a, p1, b, p2)[0]
        assert 0 <= u <= oracle.filter_pair(a, p1, b, p2)


def banks():
    from paper_0804_3643_gb300 import synth

    b1, b2 = synth.workload("plastp_plain", seed=4, scale=0.2)
    return oracle.make_bank(b1.codes, b1.seq_off), oracle.make_bank(b2.codes, b2.seq_off)


def test_gates_commute_and_shrink():
    o1, o2 = banks()
    full, pairs, through = oracle.ungapped(o1, o2, threads=8, return_pairs=True, return_filtered=True)
    assert through == pairs  # no filter
    assert (oracle.ungapped(o1, o2, oracle.Params(s0=P.s1), threads=8) == full).all()
    f = np.array([oracle.filter_pair(o1.codes[o1.seq_off[h["seq1"]]:o1.seq_off[h["seq1"] + 1]], int(h["pos1"]),
                                     o2.codes[o2.seq_off[h["seq2"]]:o2.seq_off[h["seq2"] + 1]], int(h["pos2"]))
                  for h in full])
    assert (f >= full["score"]).all()
    prev = None
    for s0 in (45, 53, 60, 80):
        got, _, n_through = oracle.ungapped(o1, o2, oracle.Params(s0=s0), threads=8, return_pairs=True,
                                            return_filtered=True)
        assert (got == full[f >= s0]).all()
        assert n_through < pairs
        if prev is not None:
            assert n_through <= prev
        prev = n_through


def test_through_count_brute_force(rng):
    # tiny banks: count the pairs with equal keys and F >= S0 one by one
    seqs1 = [rng.integers(0, 6, int(rng.integers(8, 40))).astype(np.int8) for _ in range(4)]
    seqs2 = [rng.integers(0, 6, int(rng.integers(8, 40))).astype(np.int8) for _ in range(5)]
    c1, f1 = bank_from(seqs1)
    c2, f2 = bank_from(seqs2)
    o1, o2 = oracle.make_bank(c1, f1), oracle.make_bank(c2, f2)
    for s0 in (10, 25, 40):
        want = 0
        for x in seqs1:
            for p1 in range(len(x) - 3):
                k = oracle.seed_key(x[p1:p1 + 4])
                for y in seqs2:
                    for p2 in range(len(y) - 3):
                        if k >= 0 and oracle.seed_key(y[p2:p2 + 4]) == k:
                            want += oracle.filter_pair(x, p1, y, p2) >= s0
        _, _, through = oracle.ungapped(o1, o2, oracle.Params(s0=s0), return_pairs=True, return_filtered=True)
        assert through == want
