"""Pins of the oracle's stage 2 (Section 3.3.3, the loop of Annex 4).

* identity closed form: a sequence against itself at the same seed scores
  the sum of the published BLOSUM62 diagonal over the clipped window, since
  every term is positive (the 20 residues once each sum to 116);
* hand-worked windows (negative-only, ties, clipping at both ends);
* brute force: the indexed stage 1-2 output equals all position pairs with
  equal keys scored one by one;
* symmetry under swapping the banks, and one thread equal to many.
"""
import numpy as np

import oracle
from conftest import AA, bank_from, enc, golden

P = oracle.Params()
DIAG = {a: int(v) for a, v in (x.split("=") for x in golden("blosum62_published.txt")["diagonal"].split())}


def diag_sum(codes):
    return sum(DIAG[AA[c]] for c in codes)


def test_identity_closed_form_all_twenty():
    s = enc(AA + AA)  # 40 residues, each letter twice
    # seed at 0: right window 26 cells (A..W + 6 more), left window empty
    u, rl, ll = oracle.ungapped_pair(s, 0, s, 0)
    assert u == diag_sum(s[:26]) and rl == 26 and ll == 0
    # one copy of each residue inside the right window: 116
    t = enc(AA)
    u, rl, ll = oracle.ungapped_pair(t, 0, t, 0)
    assert u == 116 and rl == 20 and ll == 0


def test_identity_closed_form_random(rng):
    for _ in range(200):
        L = int(rng.integers(4, 120))
        s = rng.integers(0, 20, L).astype(np.int8)
        p = int(rng.integers(0, L - 3))
        u, rl, ll = oracle.ungapped_pair(s, p, s, p)
        tr = min(26, L - p)
        tl = min(22, p)
        assert u == diag_sum(s[p:p + tr]) + diag_sum(s[p - tl:p])
        assert rl == tr and ll == tl


def test_hand_worked_windows():
    # all-negative right part: W vs A scores -3; maximum stays at 0
    a = enc("WWWWWWWW")
    b = enc("AAAAAAAA")
    assert oracle.ungapped_pair(a, 2, b, 2) == (0, 0, 0)
    # right: A/A=4, then W/A=-3, then A/A=4 -> running 4, 1, 5: R=5 at cell 3
    a = enc("AWA")
    b = enc("AAA")
    assert oracle.ungapped_pair(a, 0, b, 0) == (5, 3, 0)
    # a tie keeps the first maximum: 4, 1, 4 -> R=4 at cell 1 (strict >)
    a = enc("AWAP")
    b = enc("AAAA")
    # A/A 4, W/A -3, A/A 4, P/A -1  -> 4, 1, 5, 4
    assert oracle.ungapped_pair(a, 0, b, 0) == (5, 3, 0)
    a = enc("AWL")
    b = enc("AAL")
    # 4, 1, 5 -> 5 at cell 3 ... then left empty
    assert oracle.ungapped_pair(a, 0, b, 0) == (5, 3, 0)
    a = enc("AWIA")
    b = enc("AAAA")
    # A/A 4, W/A -3, I/A -1, A/A 4 -> 4, 1, 0, 4 : tie with 4, first kept
    assert oracle.ungapped_pair(a, 0, b, 0) == (4, 1, 0)
    # left part adds only when positive, the sum restarts from R:
    # seq  C A A A A  seed at 1 -> right: A/A x4 = 16 ; left: C/C = 9
    a = enc("CAAAA")
    assert oracle.ungapped_pair(a, 1, a, 1) == (25, 4, 1)
    # the running sum restarts from the right maximum, not from where the
    # right part ended: right A/A x3 = 12 then W/A -> 9; left C/C = 9 gives
    # 12 + 9 = 21 (restarting from 9 would give only 18)
    assert oracle.ungapped_pair(enc("CAAAW"), 1, enc("CAAAA"), 1) == (21, 3, 1)
    # left part negative: W/A = -3 is not added
    b = enc("WAAAA")
    c = enc("AAAAA")
    assert oracle.ungapped_pair(b, 1, c, 1) == (16, 4, 0)
    # clipping: the shorter sequence bounds both parts
    x = enc("AAAA")
    y = enc("GGAAAAGG")
    assert oracle.ungapped_pair(x, 0, y, 2) == (16, 4, 0)


def test_window_lengths_are_22_4_22():
    # 60 alanines: right part sees 26 cells, left part 22 cells
    a = enc("A" * 60)
    assert oracle.ungapped_pair(a, 30, a, 30) == (4 * 48, 26, 22)
    # shifting the other sequence keeps the clipped window sizes
    assert oracle.ungapped_pair(a, 30, a, 10) == (4 * (26 + 10), 26, 10)


def brute_ungapped(codes1, off1, codes2, off2, s1):
    out = []
    for q1 in range(len(off1) - 1):
        x = codes1[off1[q1]:off1[q1 + 1]]
        for p1 in range(len(x) - 3):
            k1 = oracle.seed_key(x[p1:p1 + 4])
            if k1 < 0:
                continue
            for q2 in range(len(off2) - 1):
                y = codes2[off2[q2]:off2[q2 + 1]]
                for p2 in range(len(y) - 3):
                    if oracle.seed_key(y[p2:p2 + 4]) != k1:
                        continue
                    u, rl, ll = oracle.ungapped_pair(x, p1, y, p2)
                    if u >= s1:
                        out.append((q1, p1, q2, p2, u, rl, ll))
    return sorted(out)


def as_tuples(h):
    return [tuple(int(v) for v in r) for r in h]


def small_banks(rng, n, lo, hi, alphabet=20, homolog=True):
    seqs = [rng.integers(0, alphabet, int(rng.integers(lo, hi))).astype(np.int8) for _ in range(n)]
    return seqs


def test_brute_force_equals_indexed(rng):
    for trial in range(4):
        s1 = small_banks(rng, 4, 5, 50, alphabet=6)  # small alphabet: many shared keys
        s2 = small_banks(rng, 5, 5, 50, alphabet=6)
        # plant a shared stretch so some pairs pass
        s2[0] = np.concatenate([s2[0], s1[0][: min(30, len(s1[0]))]])
        c1, o1 = bank_from(s1)
        c2, o2 = bank_from(s2)
        b1, b2 = oracle.make_bank(c1, o1), oracle.make_bank(c2, o2)
        for thr in (-1000, 10, 20):
            prm = oracle.Params(s1=thr)
            got = as_tuples(oracle.ungapped(b1, b2, prm))
            assert got == brute_ungapped(c1, o1, c2, o2, thr)


def test_swap_symmetry_and_threads(rng):
    from paper_0804_3643_gb300 import synth
    b1, b2 = synth.workload("plastp_plain", seed=3, scale=0.1)
    B1 = oracle.make_bank(b1.codes, b1.seq_off)
    B2 = oracle.make_bank(b2.codes, b2.seq_off)
    h12, pairs = oracle.ungapped(B1, B2, return_pairs=True)
    n1 = np.diff(B1.idx.key_off)
    n2 = np.diff(B2.idx.key_off)
    assert pairs == int((n1 * n2).sum())
    h21 = oracle.ungapped(B2, B1)
    t = h21.copy()
    t["seq1"], t["pos1"], t["seq2"], t["pos2"] = h21["seq2"], h21["pos2"], h21["seq1"], h21["pos1"]
    t = np.sort(t, order=["seq1", "pos1", "seq2", "pos2"])
    assert (t == h12).all()
    for th in (2, 5):
        assert (oracle.ungapped(B1, B2, threads=th) == h12).all()


def test_empty_banks():
    c, o = bank_from([])
    e = oracle.make_bank(c, o)
    c2, o2 = bank_from(["AQAAAQAA"])
    b = oracle.make_bank(c2, o2)
    assert len(oracle.ungapped(e, b)) == 0 and len(oracle.ungapped(b, e)) == 0
