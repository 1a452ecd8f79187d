"""Continuous-batching search service over a device-resident indexed bank.

A large protein bank is indexed once and stays in device memory.  Query
banks (requests) arrive over time; whenever a slot is free and the memory
budget allows, every waiting request (up to a batch limit) is merged into one
query bank and searched against the resident bank on that slot's CUDA stream
(plast_index_bank of the batch, then plast_search).  Slots run concurrently,
so a batch admitted while another is on the GPU overlaps with it on the
device.  Each request's records are cut out of its batch's records and
renumbered to the request's own sequence indices; since stages 1-3.1 treat
every query sequence independently (Section 5.1: the work splits per seed and
per sequence), a request's result is the same alone and in any batch.

The scheduling (admission, batching, memory accounting, latency bookkeeping)
is plain host code, independent of the executor, so it can be checked on the
CPU with a stand-in executor; ``GpuExecutor`` is the one that runs the
library.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field
from typing import Callable

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float              # seconds since the start of the run
    codes: np.ndarray           # int8 residue codes of the query bank
    seq_off: np.ndarray         # int64 offsets
    admitted: float = -1.0
    done: float = -1.0
    batch: int = -1
    result: object = None

    @property
    def n_seqs(self) -> int:
        return len(self.seq_off) - 1

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class Batch:
    bid: int
    requests: list
    mem_bytes: int
    started: float = -1.0
    finished: float = -1.0
    pairs: int = 0


def merge_queries(reqs: list) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """One query bank from several requests: (codes, seq_off, first sequence of
    each request)."""
    codes = np.concatenate([r.codes for r in reqs]) if reqs else np.zeros(0, np.int8)
    lens = np.concatenate([np.diff(r.seq_off) for r in reqs]) if reqs else np.zeros(0, np.int64)
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    first = np.zeros(len(reqs) + 1, dtype=np.int64)
    np.cumsum([r.n_seqs for r in reqs], out=first[1:])
    return codes.astype(np.int8), off, first


def split_records(recs: np.ndarray, first: np.ndarray) -> list:
    """Records (or alignments) of a merged batch, cut per request, seq1
    renumbered locally.  ``recs`` is sorted by seq1 (canonical order)."""
    out = []
    cuts = np.searchsorted(recs["seq1"], first)
    for q in range(len(first) - 1):
        part = recs[cuts[q]:cuts[q + 1]].copy()
        part["seq1"] -= first[q]
        out.append(part)
    return out


class Server:
    """Admission and dispatch.  ``execute(batch_requests)`` returns
    (per-request results, pairs) and runs on a slot thread; ``mem_of``
    estimates a batch's device memory."""

    def __init__(self, execute: Callable, mem_of: Callable, slots: int = 2, mem_budget: int = 1 << 40,
                 max_batch_seqs: int = 3000, max_batch_requests: int = 64):
        self.execute = execute
        self.mem_of = mem_of
        self.slots = slots
        self.mem_budget = mem_budget
        self.max_batch_seqs = max_batch_seqs
        self.max_batch_requests = max_batch_requests
        self.cv = threading.Condition()
        self.waiting: list[Request] = []
        self.mem_in_use = 0
        self.busy = 0
        self.batches: list[Batch] = []
        self.peak_mem = 0
        self.peak_busy = 0
        self.errors: list[BaseException] = []

    # -- batching policy: all waiting requests in arrival order, up to the
    # limits; a request larger than the limits goes alone
    def _form_batch(self) -> list:
        take, seqs = [], 0
        for r in self.waiting:
            if take and (seqs + r.n_seqs > self.max_batch_seqs or len(take) >= self.max_batch_requests):
                break
            take.append(r)
            seqs += r.n_seqs
        return take

    def _slot(self, batch: Batch, t0: float):
        try:
            res, pairs = self.execute(batch.requests)
            now = time.perf_counter() - t0
            with self.cv:
                batch.finished = now
                batch.pairs = pairs
                for r, x in zip(batch.requests, res):
                    r.result = x
                    r.done = now
        except BaseException as e:  # noqa: BLE001 - reported by run()
            with self.cv:
                self.errors.append(e)
                for r in batch.requests:
                    r.done = time.perf_counter() - t0
        finally:
            with self.cv:
                self.mem_in_use -= batch.mem_bytes
                self.busy -= 1
                self.cv.notify_all()

    def run(self, requests: list[Request], realtime: bool = True, timeout: float = 600.0) -> list[Request]:
        """Serve ``requests`` (arrival times in seconds from now).  With
        realtime=False all requests are available at once."""
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        threads = []
        nb = 0
        i = 0
        deadline = t0 + timeout
        with self.cv:
            while True:
                now = time.perf_counter() - t0
                while i < len(pending) and (not realtime or pending[i].arrival <= now):
                    self.waiting.append(pending[i])
                    i += 1
                if self.errors:
                    break
                dispatched = False
                if self.waiting and self.busy < self.slots:
                    take = self._form_batch()
                    mem = self.mem_of(take)
                    if self.mem_in_use + mem <= self.mem_budget or self.busy == 0:
                        for r in take:
                            self.waiting.remove(r)
                            r.admitted = now
                            r.batch = nb
                        b = Batch(nb, take, mem, started=now)
                        nb += 1
                        self.batches.append(b)
                        self.mem_in_use += mem
                        self.busy += 1
                        self.peak_mem = max(self.peak_mem, self.mem_in_use)
                        self.peak_busy = max(self.peak_busy, self.busy)
                        th = threading.Thread(target=self._slot, args=(b, t0), daemon=True)
                        th.start()
                        threads.append(th)
                        dispatched = True
                if i == len(pending) and not self.waiting and self.busy == 0:
                    break
                if time.perf_counter() > deadline:
                    raise TimeoutError("serving run exceeded its time limit")
                if not dispatched:
                    wait = 0.05
                    if realtime and i < len(pending):
                        wait = min(wait, max(0.0, pending[i].arrival - (time.perf_counter() - t0)))
                    self.cv.wait(timeout=max(wait, 1e-4))
        for th in threads:
            th.join()
        if self.errors:
            raise self.errors[0]
        return requests


def latency_summary(reqs: list[Request], pairs: int, wall: float) -> dict:
    lat = np.array([r.latency for r in reqs])
    return {
        "requests": len(reqs),
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_ms": float(lat.mean() * 1e3),
        "pairs_per_s": pairs / wall if wall > 0 else 0.0,
    }


class GpuExecutor:
    """Runs batches through the library against a resident bank (bank 2).
    With ``full_gapped`` a request's result is its stage-3.2 alignments
    (plast_alignment rows, drop-off ``xdrop``, kept at ``s3`` or more) rather
    than its stage-3.1 records: the redundancy lists of stage 3.2 are kept
    per pair of sequences, and a pair belongs to one request, so a request's
    alignments are the same alone and in any batch."""

    def __init__(self, codes: np.ndarray, seq_off: np.ndarray, params=None, device: int = 0,
                 full_gapped: bool = False, xdrop: int | None = None, s3: int = 47):
        import torch

        from . import binding as B

        self.B = B
        self.torch = torch
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.params = params
        d = B.DeviceBank.from_host(codes, seq_off, self.device)
        self.bank = B.plast_index_bank(d.codes, d.seq_off, params)
        self.n_resident = len(codes)
        self.full_gapped = full_gapped
        self.xdrop = B.PLAST_XDROP if xdrop is None else xdrop
        self.s3 = s3
        self._streams = threading.local()

    def _stream(self):
        s = getattr(self._streams, "s", None)
        if s is None:
            s = self.torch.cuda.Stream(device=self.device)
            self._streams.s = s
        return s

    def mem_of(self, reqs: list) -> int:
        """Device bytes a batch may hold: its index (about 70 B per residue)
        and the library's stage-2 scratch (12 B per reserved survivor, two
        copies, pairs / 128 reserved; pairs ~ 2e-4 per residue pair)."""
        res = sum(len(r.codes) for r in reqs)
        pairs = 2.1e-4 * res * self.n_resident
        mem = int(70 * res + 24 * (pairs / 128 + (1 << 20)))
        if self.full_gapped:  # stage 3.2: the warps' working space (a 1 MiB arena and
            # 96 KiB of segment lists for each of 24 warps per SM) and about 200 B per record
            n_sm = self.torch.cuda.get_device_properties(self.device).multi_processor_count
            mem += n_sm * 24 * ((1 << 20) + 3 * 8192 * 4) + int(200 * 2.5e-4 * pairs)
        return mem

    def execute(self, reqs: list):
        B, torch = self.B, self.torch
        torch.cuda.set_device(self.device)
        codes, off, first = merge_queries(reqs)
        st = self._stream()
        with torch.cuda.stream(st):
            hc = torch.from_numpy(codes).pin_memory()
            ho = torch.from_numpy(off).pin_memory()
            dc = hc.to(self.device, non_blocking=True)
            do = ho.to(self.device, non_blocking=True)
            q = B.plast_index_bank(dc, do, self.params, stream=st)
            pairs = B.plast_pair_count(q, self.bank)
            recs = B.plast_search(q, self.bank, self.params, stream=st)
            if self.full_gapped:
                al, _ = B.plast_full_gapped(q, self.bank, recs, self.params, xdrop=self.xdrop, s3=self.s3,
                                            stream=st)
                host = B.alignments_numpy(al)
            else:
                host = B.gapped_numpy(recs)
            q.free()
        return split_records(host, first), pairs

    def alone(self, req: Request):
        """The request searched on its own (reference for the batched result)."""
        return self.execute([req])[0][0]
