"""CPU oracle for PLAST's hot path (Nguyen & Lavenier, INRIA RR-6513, 2008).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_0804_3643_gb300``) never imports it and
shares no source with it.

The arithmetic lives in ``oracle.c`` (plain C, built with gcc -O2, no
intrinsics).  This module only marshals numpy arrays through ctypes.  Each
function names the passage of the paper it states; the pins that check the
oracle against facts other than itself are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

NKEYS = 8800

# Record layouts (own declarations; the product library declares its own).
HIT_DTYPE = np.dtype(
    [("seq1", "<i4"), ("pos1", "<i4"), ("seq2", "<i4"), ("pos2", "<i4"),
     ("score", "<i2"), ("rlen", "i1"), ("llen", "i1")])
GAPPED_DTYPE = np.dtype(
    [("seq1", "<i4"), ("pos1", "<i4"), ("seq2", "<i4"), ("pos2", "<i4"),
     ("score", "<i2"), ("ungapped", "<i2"), ("r_i", "<i2"), ("r_j", "<i2"),
     ("l_i", "<i2"), ("l_j", "<i2")])
assert HIT_DTYPE.itemsize == 20 and GAPPED_DTYPE.itemsize == 28
ALIGN_FIELDS = ("seq1", "seq2", "pos1", "pos2", "score", "q_start", "q_end", "s_start", "s_end", "length",
                "identities", "mismatches", "gap_opens")
ALIGN_DTYPE = np.dtype([(n, "<i4") for n in ALIGN_FIELDS])

# Stage 3.2 defaults (readings: the paper values neither): X = 38, BLAST's
# preliminary gapped drop-off of 15 bits at BLOSUM62 11/1's gapped lambda
# 0.267; S3 = S2 (E-values are out of scope).
XDROP = 38
S3 = 47


class _Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("w", "nl", "nr", "s1", "lg", "band", "gap_open", "gap_extend", "s2", "s0")]


@dataclass
class Params:
    """Method parameters.  w, nl, nr: Section 3.3.2 neighbourhoods (48-cell
    window of Annex 4 read as 22 + 4 + 22); s1, s2: thresholds of Section
    3.2; lg, band: extent of the small gapped extension of Section 3.3.4;
    gap_open / gap_extend: a gap of length k costs open + k * extend; s0:
    Section 4.2's filter threshold (0: no filter)."""
    w: int = 4
    nl: int = 22
    nr: int = 22
    s1: int = 38
    lg: int = 64
    band: int = 8
    gap_open: int = 11
    gap_extend: int = 1
    s2: int = 47
    s0: int = 0

    def c(self) -> _Params:
        return _Params(self.w, self.nl, self.nr, self.s1, self.lg, self.band,
                       self.gap_open, self.gap_extend, self.s2, self.s0)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, no intrinsics)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-shared", "-fPIC",
                               "-pthread", SRC, "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        L.oracle_score.argtypes = [ctypes.c_int, ctypes.c_int]
        L.oracle_score.restype = ctypes.c_int
        L.oracle_seed_class.argtypes = [ctypes.c_int, ctypes.c_int]
        L.oracle_seed_class.restype = ctypes.c_int
        L.oracle_seed_key.argtypes = [P]
        L.oracle_seed_key.restype = i32
        L.oracle_index.argtypes = [P, P, i32, P, P]
        L.oracle_index.restype = i64
        L.oracle_ungapped_pair.argtypes = [P, i64, i64, P, i64, i64, P, P, P]
        L.oracle_ungapped_pair.restype = i32
        L.oracle_gapped_side.argtypes = [P, i64, i32, P, i64, i32, i32, i32, i32, P, P]
        L.oracle_gapped_side.restype = i32
        L.oracle_small_gapped_pair.argtypes = [P, i64, i64, P, i64, i64, P, P, P, P, P]
        L.oracle_small_gapped_pair.restype = i32
        L.oracle_filter_pair.argtypes = [P, i64, i64, P, i64, i64, P]
        L.oracle_filter_pair.restype = i32
        L.oracle_ungapped.argtypes = [P, P, i32, P, P, P, P, i32, P, P, P, i32, i32, P, i32, P, P, P]
        L.oracle_ungapped.restype = i64
        L.oracle_small_gapped.argtypes = [P, P, P, P, P, P, i64, i32, P]
        L.oracle_xdrop_side.argtypes = [P, i64, i32, P, i64, i32, i32, i32, i32, P, P, P, P]
        L.oracle_xdrop_side.restype = i32
        L.oracle_full_gapped_one.argtypes = [P, i64, i64, P, i64, i64, i32, i32, i32, P, P, i32, P]
        L.oracle_full_gapped_one.restype = i32
        L.oracle_full_gapped.argtypes = [P, P, P, P, i32, i32, i32, i32, P, i64, i32, P, P]
        L.oracle_full_gapped.restype = i64
        L.oracle_small_gapped.restype = i64
        L.oracle_free.argtypes = [P]
        L.oracle_smith_waterman.argtypes = [P, i32, P, i32, i32, i32]
        L.oracle_smith_waterman.restype = i32
        L.oracle_codon.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.oracle_codon.restype = ctypes.c_int
        L.oracle_translate6.argtypes = [P, P, i32, P, P, P]
        L.oracle_translate6.restype = i64
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int8)


# --------------------------------------------------------------------------
# Scoring tables (Section 3.3.1, 3.3.3)
# --------------------------------------------------------------------------
def score(a: int, b: int) -> int:
    """BLOSUM62 entry for residue codes a, b (0..19, 20 = stop)."""
    return lib().oracle_score(a, b)


def blosum62() -> np.ndarray:
    return np.array([[score(a, b) for b in range(21)] for a in range(21)], dtype=np.int32)


def seed_class(position: int, aa: int) -> int:
    """Subset-seed class of residue ``aa`` at seed position 1..4 (Section 3.3.1)."""
    return lib().oracle_seed_class(position, aa)


def seed_key(word) -> int:
    w = _i8(word)
    assert w.size >= 4
    return lib().oracle_seed_key(_p(w))


# --------------------------------------------------------------------------
# Stage 0: index (Section 3.3.1)
# --------------------------------------------------------------------------
@dataclass
class Index:
    key_off: np.ndarray  # int64[8801]
    pos: np.ndarray      # int32[n], global residue index, ascending within key


def index(codes, seq_off) -> Index:
    codes = _i8(codes)
    seq_off = np.ascontiguousarray(seq_off, dtype=np.int64)
    key_off = np.zeros(NKEYS + 1, dtype=np.int64)
    pos = np.zeros(max(codes.size, 1), dtype=np.int32)
    n = lib().oracle_index(_p(codes), _p(seq_off), len(seq_off) - 1, _p(key_off), _p(pos))
    return Index(key_off, pos[:n].copy())


# --------------------------------------------------------------------------
# Stage 2: ungapped extension (Section 3.3.3, Annex 4)
# --------------------------------------------------------------------------
def ungapped_pair(s1, p1: int, s2, p2: int, params: Params = Params()):
    """(U, rlen, llen) of the hit at seed starts p1 in s1 and p2 in s2."""
    a, b = _i8(s1), _i8(s2)
    rl, ll = ctypes.c_int32(), ctypes.c_int32()
    prm = params.c()
    u = lib().oracle_ungapped_pair(_p(a), a.size, p1, _p(b), b.size, p2, ctypes.byref(prm),
                                   ctypes.byref(rl), ctypes.byref(ll))
    return u, rl.value, ll.value


def filter_pair(s1, p1: int, s2, p2: int, params: Params = Params()) -> int:
    """Section 4.2's raw score of the pair at seed starts p1, p2: the sum of
    the positive substitution scores over the ungapped window."""
    a, b = _i8(s1), _i8(s2)
    prm = params.c()
    return lib().oracle_filter_pair(_p(a), a.size, p1, _p(b), b.size, p2, ctypes.byref(prm))


@dataclass
class Bank:
    codes: np.ndarray    # int8, concatenated residues
    seq_off: np.ndarray  # int64[n_seqs + 1]
    idx: Index | None = None

    @property
    def n_seqs(self) -> int:
        return len(self.seq_off) - 1

    def indexed(self) -> "Bank":
        if self.idx is None:
            self.idx = index(self.codes, self.seq_off)
        return self


def make_bank(codes, seq_off) -> Bank:
    return Bank(_i8(codes), np.ascontiguousarray(seq_off, dtype=np.int64)).indexed()


def ungapped(b1: Bank, b2: Bank, params: Params = Params(), key_lo: int = 0, key_hi: int = NKEYS,
             threads: int = 1, return_pairs: bool = False, keys=None, return_filtered: bool = False):
    """Stages 1-2 over keys [key_lo, key_hi) (or over the key list ``keys``):
    ungapped hits with U >= s1, sorted by (seq1, pos1, seq2, pos2).  With
    params.s0 > 0, only pairs through Section 4.2's filter are extended.
    ``return_pairs`` adds the number of pairs, ``return_filtered`` the number
    of them that went through the filter."""
    b1.indexed()
    b2.indexed()
    klist = None
    if keys is not None:
        klist = np.ascontiguousarray(keys, dtype=np.int32)
        key_lo, key_hi = 0, len(klist)
    out = ctypes.c_void_p()
    pairs, filtered = ctypes.c_int64(), ctypes.c_int64()
    prm = params.c()
    L = lib()
    n = L.oracle_ungapped(_p(b1.codes), _p(b1.seq_off), b1.n_seqs, _p(b1.idx.key_off), _p(b1.idx.pos),
                          _p(b2.codes), _p(b2.seq_off), b2.n_seqs, _p(b2.idx.key_off), _p(b2.idx.pos),
                          ctypes.byref(prm), key_lo, key_hi, _p(klist) if klist is not None else None, threads,
                          ctypes.byref(out), ctypes.byref(pairs), ctypes.byref(filtered))
    buf = (ctypes.c_char * (n * HIT_DTYPE.itemsize)).from_address(out.value) if n else b""
    hits = np.frombuffer(bytes(buf), dtype=HIT_DTYPE).copy()
    L.oracle_free(out)
    res = (hits,) + ((pairs.value,) if return_pairs else ()) + ((filtered.value,) if return_filtered else ())
    return res if len(res) > 1 else hits


# --------------------------------------------------------------------------
# Stage 3.1: small gapped extension (Section 3.3.4, Section 5.2.2)
# --------------------------------------------------------------------------
def gapped_side(A, B, band: int, go: int = 11, ge: int = 1):
    """(score, end_i, end_j) of one anchored banded side (stride +1)."""
    a, b = _i8(A), _i8(B)
    ei, ej = ctypes.c_int32(), ctypes.c_int32()
    s = lib().oracle_gapped_side(_p(a), 1, a.size, _p(b), 1, b.size, band, go, ge,
                                 ctypes.byref(ei), ctypes.byref(ej))
    return s, ei.value, ej.value


def small_gapped_pair(s1, p1: int, s2, p2: int, params: Params = Params()):
    """(G, r_i, r_j, l_i, l_j) of the hit anchored at p1, p2."""
    a, b = _i8(s1), _i8(s2)
    v = [ctypes.c_int32() for _ in range(4)]
    prm = params.c()
    g = lib().oracle_small_gapped_pair(_p(a), a.size, p1, _p(b), b.size, p2, ctypes.byref(prm),
                                       *[ctypes.byref(x) for x in v])
    return (g,) + tuple(x.value for x in v)


def small_gapped(b1: Bank, b2: Bank, hits: np.ndarray, params: Params = Params(), threads: int = 1) -> np.ndarray:
    """Stage 3.1 of every hit, keeping those with G >= s2, in input order
    (``threads`` share the hits; the result does not depend on them)."""
    hits = np.ascontiguousarray(hits, dtype=HIT_DTYPE)
    out = ctypes.c_void_p()
    prm = params.c()
    L = lib()
    n = L.oracle_small_gapped(_p(b1.codes), _p(b1.seq_off), _p(b2.codes), _p(b2.seq_off), ctypes.byref(prm),
                              _p(hits) if hits.size else None, hits.size, threads, ctypes.byref(out))
    buf = (ctypes.c_char * (n * GAPPED_DTYPE.itemsize)).from_address(out.value) if n else b""
    res = np.frombuffer(bytes(buf), dtype=GAPPED_DTYPE).copy()
    L.oracle_free(out)
    return res


# --------------------------------------------------------------------------
# Stage 3.2 and the tabular fields of stage 4 (Sections 3.3.4, 3.3.5)
# --------------------------------------------------------------------------
def xdrop_side(A, B, go: int = 11, ge: int = 1, x: int = XDROP):
    """(score, end_i, end_j, path) of one anchored, unbanded side with the
    row-wise drop-off x; path is a string of M / I / D from the anchor out."""
    a, b = _i8(A), _i8(B)
    ei, ej, nops = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ops = ctypes.create_string_buffer(a.size + b.size + 1)
    sc = lib().oracle_xdrop_side(_p(a), 1, a.size, _p(b), 1, b.size, go, ge, x, ctypes.byref(ei), ctypes.byref(ej),
                                 ops, ctypes.byref(nops))
    return sc, ei.value, ej.value, ops.raw[: nops.value].decode()


def full_gapped_one(s1, p1: int, s2, p2: int, go: int = 11, ge: int = 1, x: int = XDROP):
    """(alignment record, [(diagonal, start, stop), ...]) of the full gapped
    extension anchored at seed starts p1, p2 (seq1 / seq2 fields left 0)."""
    a, b = _i8(s1), _i8(s2)
    al = np.zeros(1, dtype=ALIGN_DTYPE)
    cap = a.size + b.size + 4
    segs = np.zeros(3 * cap, dtype=np.int32)
    nseg = ctypes.c_int32()
    lib().oracle_full_gapped_one(_p(a), a.size, p1, _p(b), b.size, p2, go, ge, x, _p(al), _p(segs), cap,
                                 ctypes.byref(nseg))
    return al[0], [tuple(int(v) for v in segs[3 * k: 3 * k + 3]) for k in range(nseg.value)]


def full_gapped(b1: Bank, b2: Bank, records: np.ndarray, params: Params = Params(), x: int = XDROP, s3: int = S3,
                threads: int = 1, return_extended: bool = False):
    """Stage 3.2 of stage-3.1 records (any order) with the redundancy lists:
    alignments scoring >= s3, sorted by (seq1, pos1, seq2, pos2) of their
    anchors; ``return_extended`` adds how many records were extended."""
    recs = np.ascontiguousarray(records, dtype=GAPPED_DTYPE)
    out = ctypes.c_void_p()
    ext = ctypes.c_int64()
    L = lib()
    n = L.oracle_full_gapped(_p(b1.codes), _p(b1.seq_off), _p(b2.codes), _p(b2.seq_off), params.gap_open,
                             params.gap_extend, x, s3, _p(recs) if recs.size else None, recs.size, threads,
                             ctypes.byref(out), ctypes.byref(ext))
    buf = (ctypes.c_char * (n * ALIGN_DTYPE.itemsize)).from_address(out.value) if n else b""
    res = np.frombuffer(bytes(buf), dtype=ALIGN_DTYPE).copy()
    L.oracle_free(out)
    return (res, ext.value) if return_extended else res


def search(b1: Bank, b2: Bank, params: Params = Params(), threads: int = 1) -> np.ndarray:
    """Stages 0-3.1 of Section 3.2: ungapped hits, then small gapped >= s2."""
    return small_gapped(b1, b2, ungapped(b1, b2, params, threads=threads), params)


def smith_waterman(a, b, go: int = 11, ge: int = 1) -> int:
    x, y = _i8(a), _i8(b)
    return lib().oracle_smith_waterman(_p(x), x.size, _p(y), y.size, go, ge)


# --------------------------------------------------------------------------
# Six-frame translation (Section 6)
# --------------------------------------------------------------------------
def codon(n1: int, n2: int, n3: int) -> int:
    return lib().oracle_codon(n1, n2, n3)


def translate6(dna, contig_off):
    """(aa codes int8, seq_off int64[6n+1], meta int32[6n, 2]) of the six frames."""
    d = np.ascontiguousarray(dna, dtype=np.uint8)
    off = np.ascontiguousarray(contig_off, dtype=np.int64)
    n = len(off) - 1
    aa = np.zeros(max(2 * d.size, 1), dtype=np.int8)
    seq_off = np.zeros(6 * n + 1, dtype=np.int64)
    meta = np.zeros(12 * n, dtype=np.int32)
    m = lib().oracle_translate6(_p(d), _p(off), n, _p(aa), _p(seq_off), _p(meta))
    return aa[:m].copy(), seq_off, meta.reshape(-1, 2)
