"""Pins of the oracle's tables against published facts (not against itself).

* BLOSUM62: symmetry, the published diagonal and extremes, and NCBI's
  Karlin-Altschul lambda and H recomputed from the transcribed matrix.
* Subset seed (Section 3.3.1): every letter in exactly one class per
  position, class counts 20 / 2 / 11 / 20, the printed AQAA/APAA/ASAA
  example, and a one-to-one key numbering.
* Genetic code (Section 6 translation): degeneracies, stops, known codons.
"""
import itertools

import numpy as np
import pytest

import oracle
from conftest import AA, enc, golden
from paper_0804_3643_gb300 import synth


def test_blosum62_symmetric_and_diagonal():
    B = oracle.blosum62()
    assert (B == B.T).all()
    g = golden("blosum62_published.txt")
    diag = dict(x.split("=") for x in g["diagonal"].split())
    for a, v in diag.items():
        assert B[AA.index(a), AA.index(a)] == int(v), a
    assert sum(int(v) for v in diag.values()) == 116
    assert B[:20, :20].min() == int(g["min"])
    assert B[:20, :20].max() == int(g["max"])
    # stop row: -4 against residues, +1 against itself
    assert (B[20, :20] == -4).all() and B[20, 20] == 1


def test_blosum62_karlin_altschul_constants():
    """lambda and H recomputed from the transcribed matrix and the Robinson &
    Robinson background match NCBI's published 0.3176 and 0.4012; a wrong
    entry of a common pair moves them visibly."""
    g = golden("blosum62_published.txt")
    S = oracle.blosum62()[:20, :20].astype(np.float64)
    p = synth.RR_FREQ
    P = p[:, None] * p[None, :]
    assert (P * S).sum() < 0  # negative expected score: local statistics apply

    def f(lam):
        return (P * np.exp(lam * S)).sum() - 1.0

    lo, hi = 1e-4, 3.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (lo, mid) if f(mid) > 0 else (mid, hi)
    lam = 0.5 * (lo + hi)
    H = lam * (P * S * np.exp(lam * S)).sum()
    assert abs(lam - float(g["lambda"])) < 1e-4
    assert abs(H - float(g["H"])) < 1e-4


def _classes(pos):
    return {a: oracle.seed_class(pos, AA.index(a)) for a in AA}


def test_subset_seed_classes_match_paper_table():
    g = golden("subset_seed.txt")
    for pos in (1, 2, 3, 4):
        groups = []
        for tok in g[f"position {pos}"].split():
            groups.append(tok.strip("{}"))
        # every letter appears in exactly one printed group
        letters = "".join(groups)
        assert sorted(letters) == sorted(AA), pos
        cls = _classes(pos)
        # letters of one printed group share a class, different groups differ
        ids = [{cls[a] for a in grp} for grp in groups]
        assert all(len(s) == 1 for s in ids), pos
        assert len({next(iter(s)) for s in ids}) == len(groups), pos
    assert [len(set(_classes(p).values())) for p in (1, 2, 3, 4)] == [20, 2, 11, 20]
    # the stop and codes outside the alphabet have no class
    assert all(oracle.seed_class(p, 20) == -1 for p in (1, 2, 3, 4))


def test_subset_seed_printed_example():
    g = golden("subset_seed.txt")
    words = g["same key"].split()
    keys = {oracle.seed_key(enc(w)) for w in words}
    assert len(keys) == 1
    # a class-2 'c' letter (C) at position 2 gives another key
    assert oracle.seed_key(enc("ACAA")) not in keys
    # and so do different singletons at positions 1 and 4
    assert oracle.seed_key(enc("RQAA")) not in keys
    assert oracle.seed_key(enc("AQAR")) not in keys


def test_seed_key_is_a_bijection_on_class_tuples():
    reps = [{}, {}, {}, {}]
    for p in range(4):
        for a in range(20):
            reps[p].setdefault(oracle.seed_class(p + 1, a), a)
    keys = set()
    for combo in itertools.product(*[sorted(r.values()) for r in reps]):
        k = oracle.seed_key(np.array(combo, dtype=np.int8))
        assert 0 <= k < oracle.NKEYS
        keys.add(k)
    assert len(keys) == 20 * 2 * 11 * 20 == oracle.NKEYS
    assert oracle.seed_key(enc("AQ*A")) == -1


def test_genetic_code():
    g = golden("genetic_code.txt")
    nt = {"A": 0, "C": 1, "G": 2, "T": 3}
    table = {}
    for c in itertools.product("ACGT", repeat=3):
        table["".join(c)] = oracle.codon(*[nt[x] for x in c])
    stops = sorted(k for k, v in table.items() if v == 20)
    assert stops == sorted(g["stops"].split())
    counts = {}
    for v in table.values():
        if v != 20:
            counts[AA[v]] = counts.get(AA[v], 0) + 1
    want = dict(x.split("=") for x in g["degeneracy"].split())
    assert counts == {k: int(v) for k, v in want.items()}
    assert sum(counts.values()) == 61
    for kv in g["codons"].split():
        cod, aa = kv.split("=")
        assert table[cod] == AA.index(aa), cod
