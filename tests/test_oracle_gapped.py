"""Pins of the oracle's stage 3.1 (Section 3.3.4, Section 5.2.2).

* band-0 reduction: with no room for gaps the small gapped score equals the
  ungapped score over windows of lg residues on each side;
* hand-worked sides (affine gap cost, end-cell tie rule);
* single-gap closed form: an identical stretch with one deleted residue;
* Smith-Waterman (textbook Gotoh local alignment): an upper bound for every
  hit, and on tiny inputs with unbounded band the maximum over all anchors
  equals it exactly;
* gapped >= ungapped for every hit; symmetry under swapping the sequences.
"""
import numpy as np
import pytest

import oracle
from conftest import AA, bank_from, enc, golden

DIAG = {a: int(v) for a, v in (x.split("=") for x in golden("blosum62_published.txt")["diagonal"].split())}


def test_hand_worked_sides():
    assert oracle.gapped_side(enc("WWW"), enc("WWW"), band=8) == (33, 3, 3)
    assert oracle.gapped_side(enc("W"), enc(""), band=8) == (0, 0, 0)
    assert oracle.gapped_side(enc(""), enc(""), band=8) == (0, 0, 0)
    # one inserted G in B: gap path 55 - 12 + 55 = 98 beats the mismatch
    # path 55 - 2 + 44 = 97
    a = enc("W" * 10)
    b = enc("W" * 5 + "G" + "W" * 5)
    assert oracle.gapped_side(a, b, band=8) == (98, 10, 11)
    # band 0 forbids the gap: the mismatch path is the best left
    assert oracle.gapped_side(a, b, band=0) == (97, 10, 10)
    # a two-residue gap costs 11 + 2 = 13: 55 - 13 + 55 = 97 vs mismatch
    # path 55 - 2 - 2 + 33 = 84 (W/G = -2)
    b2 = enc("W" * 5 + "GG" + "W" * 5)
    assert oracle.gapped_side(a, b2, band=8) == (97, 10, 12)
    # tie rule: the first maximum in row-major order wins.  On "AWPA" vs
    # "AAAA" the diagonal runs A/A 4, W/A -3, P/A -1, A/A 4 -> 4, 1, 0, 4 and
    # every gapped path costs at least 12, so 4 is reached at (1,1) and again
    # at (4,4); (1,1) is kept.
    assert oracle.gapped_side(enc("AWPA"), enc("AAAA"), band=8) == (4, 1, 1)
    # "AWA" vs "AAA": 4, 1, 5 -> the unique best is (3,3)
    assert oracle.gapped_side(enc("AWA"), enc("AAA"), band=8) == (5, 3, 3)


def test_band_zero_reduces_to_ungapped(rng):
    for _ in range(200):
        L1, L2 = int(rng.integers(4, 150)), int(rng.integers(4, 150))
        x = rng.integers(0, 20, L1).astype(np.int8)
        y = rng.integers(0, 20, L2).astype(np.int8)
        p1, p2 = int(rng.integers(0, L1 - 3)), int(rng.integers(0, L2 - 3))
        lg = int(rng.integers(4, 70))
        g = oracle.small_gapped_pair(x, p1, y, p2, oracle.Params(band=0, lg=lg))
        u, rl, ll = oracle.ungapped_pair(x, p1, y, p2, oracle.Params(nl=lg, nr=lg - 4))
        assert g == (u, rl, rl, ll, ll)


def test_single_gap_closed_form(rng):
    for _ in range(20):
        x = rng.integers(0, 20, 60).astype(np.int8)
        y = np.delete(x, 40)
        g, ri, rj, li, lj = oracle.small_gapped_pair(x, 0, y, 0)
        expect = sum(DIAG[AA[c]] for c in np.delete(x, 40)) - 12
        assert (g, ri, rj, li, lj) == (expect, 60, 59, 0, 0)


def test_smith_waterman_textbook():
    assert oracle.smith_waterman(enc("WWW"), enc("AWWWA")) == 33
    assert oracle.smith_waterman(enc("AAA"), enc("WWW")) == 0
    # local: the best piece only; gap costs 12 for one residue
    assert oracle.smith_waterman(enc("W" * 10), enc("W" * 5 + "G" + "W" * 5)) == 98


def test_smith_waterman_equals_max_over_anchors(rng):
    prm = oracle.Params(lg=64, band=64)
    for _ in range(40):
        x = rng.integers(0, 6, int(rng.integers(4, 14))).astype(np.int8)
        y = rng.integers(0, 6, int(rng.integers(4, 14))).astype(np.int8)
        best = max(oracle.small_gapped_pair(x, i, y, j, prm)[0] for i in range(len(x)) for j in range(len(y)))
        assert best == oracle.smith_waterman(x, y)


@pytest.fixture(scope="module")
def plain_hits():
    from paper_0804_3643_gb300 import synth
    b1, b2 = synth.workload("plastp_plain", seed=5, scale=0.1)
    B1 = oracle.make_bank(b1.codes, b1.seq_off)
    B2 = oracle.make_bank(b2.codes, b2.seq_off)
    return B1, B2, oracle.ungapped(B1, B2)


def test_bounds_on_hits(plain_hits):
    B1, B2, hits = plain_hits
    assert len(hits) > 50
    g = oracle.small_gapped(B1, B2, hits, oracle.Params(s2=-10 ** 6))
    assert len(g) == len(hits)
    assert (g["score"] >= g["ungapped"]).all()  # gapped >= ungapped
    sel = np.random.default_rng(0).choice(len(hits), size=min(150, len(hits)), replace=False)
    for k in sel:
        r = g[k]
        x = B1.codes[B1.seq_off[r["seq1"]]:B1.seq_off[r["seq1"] + 1]]
        y = B2.codes[B2.seq_off[r["seq2"]]:B2.seq_off[r["seq2"] + 1]]
        assert r["score"] <= oracle.smith_waterman(x, y)
        # swapping the two sequences leaves the score unchanged
        assert oracle.small_gapped_pair(y, int(r["pos2"]), x, int(r["pos1"]))[0] == r["score"]
        # end cells lie inside the band and the clipped windows
        assert abs(int(r["r_i"]) - int(r["r_j"])) <= 8 and abs(int(r["l_i"]) - int(r["l_j"])) <= 8
        assert r["r_i"] <= min(64, len(x) - r["pos1"]) and r["l_i"] <= min(64, r["pos1"])


def test_threshold_filter(plain_hits):
    B1, B2, hits = plain_hits
    allg = oracle.small_gapped(B1, B2, hits, oracle.Params(s2=-10 ** 6))
    kept = oracle.small_gapped(B1, B2, hits, oracle.Params(s2=47))
    assert (kept == allg[allg["score"] >= 47]).all()


def test_threads_equal_one_thread(plain_hits):
    # the hits cut into ranges over several threads give the same records in
    # the same (input) order as one thread
    B1, B2, hits = plain_hits
    many = np.concatenate([hits] * 8)
    one = oracle.small_gapped(B1, B2, many, oracle.Params(s2=30))
    assert len(one) > 0
    for th in (2, 3, 8):
        assert np.array_equal(oracle.small_gapped(B1, B2, many, oracle.Params(s2=30), threads=th).view(np.uint8),
                              one.view(np.uint8))
