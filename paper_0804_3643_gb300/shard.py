"""Sharding a comparison across processes (one GPU each).

Stages 1-3.1 treat every pair of sequences independently (Section 5.1: the
work splits per seed and, equally, per bank-2 sequence range), so a bank-2
split into contiguous sequence ranges gives each rank an independent search
against the whole bank 1; no data moves between ranks until the records are
gathered.  The records of a shard number bank-2 sequences from the shard's
first one; merging renumbers them and restores the canonical order
(seq1, pos1, seq2, pos2).  Stage 3.2 shards the same way: its redundancy
lists are kept per pair of sequences, and a pair lies in one shard, so each
rank extends its own records and the alignments merge like the records.
Plain host code: the per-rank work is the library's plast_search (and
plast_full_gapped) on that rank's GPU.
"""
from __future__ import annotations

import numpy as np


def shard_range(seq_off: np.ndarray, rank: int, world: int) -> tuple[int, int]:
    """Sequences [lo, hi) of rank's shard: contiguous ranges holding about the
    same number of residues."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    n = len(seq_off) - 1
    total = int(seq_off[-1])
    cuts = [0] + [int(np.searchsorted(seq_off, total * r / world, side="left")) for r in range(1, world)] + [n]
    cuts = [min(max(c, 0), n) for c in cuts]
    for r in range(1, world + 1):
        cuts[r] = max(cuts[r], cuts[r - 1])
    return cuts[rank], cuts[rank + 1]


def shard_bank(codes: np.ndarray, seq_off: np.ndarray, rank: int, world: int):
    """(codes, seq_off, first sequence) of rank's shard of a bank."""
    lo, hi = shard_range(seq_off, rank, world)
    a, b = int(seq_off[lo]), int(seq_off[hi])
    return codes[a:b], (seq_off[lo:hi + 1] - a).astype(np.int64), lo


def merge_records(parts: list) -> np.ndarray:
    """Records (plast_gapped) or alignments (plast_alignment) of all shards,
    as (rows, first bank-2 sequence) pairs, in canonical order with global
    bank-2 sequence numbers."""
    recs = []
    for r, first in parts:
        r = np.array(r, copy=True)
        if len(r):
            r["seq2"] += first
        recs.append(r)
    if not recs:
        raise ValueError("no shards")
    allr = np.concatenate(recs)
    order = np.lexsort((allr["pos2"], allr["seq2"], allr["pos1"], allr["seq1"]))
    return allr[order]
