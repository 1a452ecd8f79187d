"""Seeded synthetic banks standing in for the paper's PIR / SWISS-PROT /
GenBank banks (Annex 1), which are not available here.

This module only draws random inputs.  It holds none of the method's
arithmetic: no seed classes, no scoring, no extension.  Both the CUDA path
and the CPU oracle are fed from it, and nothing else is shared between them.

Input model (the same for every workload; all draws from numpy's PCG64 with
an explicit seed):

* protein lengths: lognormal with median 300 and sigma 0.45 on log(length),
  rounded and clipped to 50..1000;
* residues: i.i.d. from the Robinson & Robinson (1991) background
  frequencies, as codes 0..19 in the order A R N D C Q E G H I L K M F P S T W Y V;
* planted homologs: a copy of a bank1 protein at identity U[0.4, 0.9];
  a substituted residue a becomes b != a with probability proportional to
  p_b * 2^(s_ab / 2), s being BLOSUM62 in half-bit units (the table below is
  this generator's own copy, used only to draw substitutions); indel events
  at rate 0.02 per residue, insertion or deletion with probability 1/2,
  length 1 + Geometric(1/2) capped at 10;
* low-complexity runs: a span of U[20, 200] residues overwritten with 2-3
  residue types drawn uniformly;
* DNA: contigs of U[1, 100] kbp up to the requested total, P(A) = P(T) =
  0.275, P(C) = P(G) = 0.225 (GC 45 %), codes A C G T = 0 1 2 3; planted
  coding regions are mutated bank1 proteins back-translated with uniformly
  drawn synonymous codons, on a random strand, at non-overlapping offsets.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

AA = "ARNDCQEGHILKMFPSTWYV"

# Robinson & Robinson (1991) amino acid background frequencies.
RR_FREQ = np.array([
    0.07805, 0.05129, 0.04487, 0.05364, 0.01925, 0.04264, 0.06295, 0.07377, 0.02199, 0.05142,
    0.09019, 0.05744, 0.02243, 0.03856, 0.05203, 0.07120, 0.05841, 0.01330, 0.03216, 0.06441])
RR_FREQ = RR_FREQ / RR_FREQ.sum()

# BLOSUM62 lower triangle, rows in the order of AA; used only to weight
# substitutions when planting homologs.
_B62_LOWER = """
4
-1 5
-2 0 6
-2 -2 1 6
0 -3 -3 -3 9
-1 1 0 0 -3 5
-1 0 0 2 -4 2 5
0 -2 0 -1 -3 -2 -2 6
-2 0 1 -1 -3 0 0 -2 8
-1 -3 -3 -3 -1 -3 -3 -4 -3 4
-1 -2 -3 -4 -1 -2 -3 -4 -3 2 4
-1 2 0 -1 -3 1 1 -2 -1 -3 -2 5
-1 -1 -2 -3 -1 0 -2 -3 -2 1 2 -1 5
-2 -3 -3 -3 -2 -3 -3 -3 -1 0 0 -3 0 6
-1 -2 -2 -1 -3 -1 -1 -2 -2 -3 -3 -1 -2 -4 7
1 -1 1 0 -1 0 0 0 -1 -2 -2 0 -1 -2 -1 4
0 -1 0 -1 -1 -1 -1 -2 -2 -1 -1 -1 -1 -2 -1 1 5
-3 -3 -4 -4 -2 -2 -3 -2 -2 -3 -2 -3 -1 1 -4 -3 -2 11
-2 -2 -2 -3 -2 -1 -2 -3 2 -1 -1 -2 -1 3 -3 -2 -2 2 7
0 -3 -3 -3 -1 -2 -2 -3 -3 3 1 -2 1 -1 -2 -2 0 -3 -1 4
"""


def _substitution_cdf() -> np.ndarray:
    rows = [list(map(int, r.split())) for r in _B62_LOWER.strip().splitlines()]
    s = np.zeros((20, 20))
    for i, r in enumerate(rows):
        for j, v in enumerate(r):
            s[i, j] = s[j, i] = v
    w = RR_FREQ[None, :] * np.power(2.0, s / 2.0)
    np.fill_diagonal(w, 0.0)
    w /= w.sum(axis=1, keepdims=True)
    return np.cumsum(w, axis=1)


_SUB_CDF = _substitution_cdf()

# Synonymous codons of every amino acid under the standard genetic code, used
# only for back-translation of planted proteins (nucleotides A C G T = 0 1 2 3).
_CODONS = {
    "A": ["GCT", "GCC", "GCA", "GCG"], "R": ["CGT", "CGC", "CGA", "CGG", "AGA", "AGG"],
    "N": ["AAT", "AAC"], "D": ["GAT", "GAC"], "C": ["TGT", "TGC"], "Q": ["CAA", "CAG"],
    "E": ["GAA", "GAG"], "G": ["GGT", "GGC", "GGA", "GGG"], "H": ["CAT", "CAC"],
    "I": ["ATT", "ATC", "ATA"], "L": ["TTA", "TTG", "CTT", "CTC", "CTA", "CTG"],
    "K": ["AAA", "AAG"], "M": ["ATG"], "F": ["TTT", "TTC"], "P": ["CCT", "CCC", "CCA", "CCG"],
    "S": ["TCT", "TCC", "TCA", "TCG", "AGT", "AGC"], "T": ["ACT", "ACC", "ACA", "ACG"],
    "W": ["TGG"], "Y": ["TAT", "TAC"], "V": ["GTT", "GTC", "GTA", "GTG"],
}
_NT = {"A": 0, "C": 1, "G": 2, "T": 3}
_CODON_TAB = np.full((20, 6, 3), -1, dtype=np.int8)
_CODON_N = np.zeros(20, dtype=np.int64)
for _i, _a in enumerate(AA):
    _CODON_N[_i] = len(_CODONS[_a])
    for _k, _c in enumerate(_CODONS[_a]):
        _CODON_TAB[_i, _k] = [_NT[x] for x in _c]

DNA_FREQ = np.array([0.275, 0.225, 0.225, 0.275])  # A C G T


@dataclass
class SynthBank:
    """Concatenated int8 codes plus int64 offsets (n_seqs + 1)."""
    codes: np.ndarray
    seq_off: np.ndarray
    planted: dict = field(default_factory=dict)

    @property
    def n_seqs(self) -> int:
        return len(self.seq_off) - 1

    def seq(self, i: int) -> np.ndarray:
        return self.codes[self.seq_off[i]:self.seq_off[i + 1]]


def protein_lengths(rng: np.random.Generator, n: int, median: float = 300.0, sigma: float = 0.45,
                    lo: int = 50, hi: int = 1000) -> np.ndarray:
    x = np.exp(np.log(median) + sigma * rng.standard_normal(n))
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def background_residues(rng: np.random.Generator, n: int) -> np.ndarray:
    cdf = np.cumsum(RR_FREQ)
    out = np.empty(n, dtype=np.int8)
    step = 1 << 24
    for s in range(0, n, step):
        u = rng.random(min(step, n - s))
        out[s:s + len(u)] = np.minimum(np.searchsorted(cdf, u, side="right"), 19)
    return out


def _geometric_len(rng: np.random.Generator) -> int:
    return int(min(1 + rng.geometric(0.5) - 1, 10))


def mutate(rng: np.random.Generator, seq: np.ndarray, identity: float, indel_rate: float = 0.02) -> np.ndarray:
    """A homolog of ``seq``: substitutions at rate 1 - identity, then indels."""
    s = seq.copy()
    sub = rng.random(len(s)) >= identity
    if sub.any():
        u = rng.random(int(sub.sum()))
        cdf = _SUB_CDF[s[sub].astype(np.int64)]
        s[sub] = np.minimum((cdf < u[:, None]).sum(axis=1), 19).astype(np.int8)
    events = np.nonzero(rng.random(len(s)) < indel_rate)[0]
    if len(events) == 0:
        return s
    pieces, last = [], 0
    for e in events:
        if e < last:
            continue
        pieces.append(s[last:e])
        length = _geometric_len(rng)
        if rng.random() < 0.5:  # insertion before e
            pieces.append(background_residues(rng, length))
            last = e
        else:  # deletion of s[e : e + length]
            last = min(e + length, len(s))
    pieces.append(s[last:])
    out = np.concatenate(pieces)
    return out if len(out) >= 8 else s


def low_complexity(rng: np.random.Generator, seq: np.ndarray) -> np.ndarray:
    s = seq.copy()
    length = int(min(rng.integers(20, 201), len(s)))
    start = int(rng.integers(0, len(s) - length + 1))
    kinds = rng.choice(20, size=int(rng.integers(2, 4)), replace=False).astype(np.int8)
    s[start:start + length] = kinds[rng.integers(0, len(kinds), length)]
    return s


def _pack(seqs) -> SynthBank:
    lens = np.array([len(x) for x in seqs], dtype=np.int64)
    off = np.zeros(len(seqs) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    codes = np.concatenate(seqs).astype(np.int8) if seqs else np.zeros(0, np.int8)
    return SynthBank(codes, off)


def random_protein_bank(rng: np.random.Generator, n: int) -> SynthBank:
    lens = protein_lengths(rng, n)
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return SynthBank(background_residues(rng, int(off[-1])), off)


def protein_bank(rng: np.random.Generator, n: int, homolog_source: SynthBank | None = None,
                 planted_frac: float = 0.0, lowcomplex_frac: float = 0.0) -> SynthBank:
    """n background proteins; a fraction replaced by homologs of ``homolog_source``
    entries, a fraction carrying a low-complexity run."""
    base = random_protein_bank(rng, n)
    n_plant = int(round(planted_frac * n)) if homolog_source is not None else 0
    n_low = int(round(lowcomplex_frac * n))
    if n_plant == 0 and n_low == 0:
        return base
    seqs = [base.seq(i) for i in range(n)]
    where = rng.choice(n, size=n_plant, replace=False) if n_plant else np.zeros(0, np.int64)
    src = rng.integers(0, homolog_source.n_seqs, size=n_plant) if n_plant else np.zeros(0, np.int64)
    for i, j in zip(where, src):
        seqs[i] = mutate(rng, homolog_source.seq(int(j)), float(rng.uniform(0.4, 0.9)))
    low = rng.choice(n, size=n_low, replace=False) if n_low else np.zeros(0, np.int64)
    for i in low:
        seqs[i] = low_complexity(rng, seqs[i])
    bank = _pack(seqs)
    bank.planted = {"bank2_index": where.astype(np.int64), "bank1_source": src.astype(np.int64),
                    "low_complexity": np.sort(low).astype(np.int64)}
    return bank


def back_translate(rng: np.random.Generator, protein: np.ndarray) -> np.ndarray:
    pick = (rng.random(len(protein)) * _CODON_N[protein]).astype(np.int64)
    return _CODON_TAB[protein.astype(np.int64), pick].reshape(-1).astype(np.uint8)


def dna_bank(rng: np.random.Generator, total_nt: int, proteins: SynthBank | None = None, n_planted: int = 0,
             min_contig: int = 1000, max_contig: int = 100000) -> SynthBank:
    """Contigs of U[min, max] nt up to total_nt; n_planted back-translated
    homologs of ``proteins`` entries written at non-overlapping offsets."""
    lens = []
    acc = 0
    while acc < total_nt:
        L = int(rng.integers(min_contig, max_contig + 1))
        L = min(L, total_nt - acc) if total_nt - acc >= min_contig else L
        lens.append(L)
        acc += L
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(np.array(lens, dtype=np.int64), out=off[1:])
    cdf = np.cumsum(DNA_FREQ)
    nt = np.empty(int(off[-1]), dtype=np.uint8)
    step = 1 << 24
    for s in range(0, len(nt), step):
        u = rng.random(min(step, len(nt) - s))
        nt[s:s + len(u)] = np.minimum(np.searchsorted(cdf, u, side="right"), 3)
    used = [[] for _ in lens]
    placed = []
    for _ in range(n_planted if proteins is not None else 0):
        j = int(rng.integers(0, proteins.n_seqs))
        region = back_translate(rng, mutate(rng, proteins.seq(j), float(rng.uniform(0.4, 0.9))))
        strand = int(rng.integers(0, 2))
        if strand:  # reverse complement
            region = (3 - region[::-1]).astype(np.uint8)
        for _try in range(50):
            c = int(rng.integers(0, len(lens)))
            if lens[c] <= len(region):
                continue
            st = int(rng.integers(0, lens[c] - len(region)))
            en = st + len(region)
            if all(en <= a or st >= b for a, b in used[c]):
                used[c].append((st, en))
                nt[off[c] + st:off[c] + en] = region
                placed.append((j, c, st, strand, len(region)))
                break
    bank = SynthBank(nt.view(np.int8), off)
    bank.codes = nt
    # (source protein, contig, first nt, strand (1: reverse complement), nt)
    bank.planted = {"regions": np.array(placed, dtype=np.int64).reshape(-1, 5)}
    return bank


# --------------------------------------------------------------------------
# Named workloads.  ``scale`` shrinks the bank sizes for quick tests while
# keeping the composition model.
# --------------------------------------------------------------------------
WORKLOADS = {
    "plastp_plain": dict(n1=200, n2=2000, planted=0.10, lowc=0.0),
    "plastp_full": dict(n1=10000, n2=100000, planted=0.05, lowc=0.0),
    "batching_stress": dict(n1=50000, n2=50000, planted=0.0, lowc=0.20),
}


def workload(name: str, seed: int = 1, scale: float = 1.0, n2: int | None = None):
    """(bank1, bank2) of a named protein-vs-protein workload; ``n2`` overrides
    the number of bank-2 proteins (bank 1 is drawn first, so it is unchanged)."""
    rng = np.random.default_rng(seed)
    cfg = WORKLOADS[name]
    n1 = max(2, int(round(cfg["n1"] * scale)))
    n2 = max(2, int(round(cfg["n2"] * scale))) if n2 is None else int(n2)
    b1 = protein_bank(rng, n1, lowcomplex_frac=cfg["lowc"])
    b2 = protein_bank(rng, n2, homolog_source=b1, planted_frac=cfg["planted"], lowcomplex_frac=cfg["lowc"])
    return b1, b2


def tplastn_workload(seed: int = 1, scale: float = 1.0):
    """(protein bank1, DNA bank) of the protein-vs-translated-DNA workload:
    5,000 proteins vs 50 Mbp carrying 2,000 planted coding regions."""
    rng = np.random.default_rng(seed)
    n1 = max(2, int(round(5000 * scale)))
    b1 = protein_bank(rng, n1)
    total = max(3000, int(round(50_000_000 * scale)))
    dna = dna_bank(rng, total, proteins=b1, n_planted=max(1, int(round(2000 * scale))),
                   max_contig=max(1000, min(100000, total // 4)))
    return b1, dna


def plastx_workload(seed: int = 1, scale: float = 1.0):
    """(query DNA bank, subject DNA bank) of the translated-vs-translated
    workload: 1,000 sequences of 600-1,450 nt (mean about 1,024, the size of
    the smallest query bank of the PLAST-X runs) against 50 Mbp in sequences
    of 1-10 kbp (mean about 5.5 kbp, a third of their subject bank); both
    carry back-translated homologs of 2,000 hidden source proteins of median
    length 200 (200 planted in the queries, 2,000 in the subject)."""
    rng = np.random.default_rng(seed)
    n_src = max(2, int(round(2000 * scale)))
    lens = protein_lengths(rng, n_src, median=200.0)
    off = np.zeros(n_src + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    src = SynthBank(background_residues(rng, int(off[-1])), off)
    n_q = max(2, int(round(1000 * scale)))
    query = dna_bank(rng, n_q * 1024, proteins=src, n_planted=max(1, int(round(200 * scale))),
                     min_contig=600, max_contig=1450)
    total = max(12000, int(round(50_000_000 * scale)))
    subject = dna_bank(rng, total, proteins=src, n_planted=max(1, int(round(2000 * scale))),
                       min_contig=1000, max_contig=10000)
    return query, subject


def serving_requests(seed: int, n: int, rate_per_s: float, max_proteins: int = 500):
    """Poisson arrivals: list of (arrival time s, SynthBank query)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    out = []
    for i in range(n):
        k = int(rng.integers(1, max_proteins + 1))
        out.append((float(t[i]), random_protein_bank(rng, k)))
    return out
