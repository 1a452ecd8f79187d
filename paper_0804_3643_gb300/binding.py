"""Python binding of the C ABI in include/plast.h (ctypes; argument marshalling
only).  Every function keeps the C name.  Device memory and streams come from
PyTorch; every computation runs in libplast.so's CUDA kernels.  There is no
CPU path: if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

LIB_PATH = _build.LIB

PLAST_OK = 0
PLAST_E_INVALID = -1
PLAST_E_OOM = -2
PLAST_E_CAPACITY = -3
PLAST_E_CUDA = -4
PLAST_E_TIMEOUT = -5
NKEYS = 8800

HIT_DTYPE = np.dtype(
    [("seq1", "<i4"), ("pos1", "<i4"), ("seq2", "<i4"), ("pos2", "<i4"),
     ("score", "<i2"), ("rlen", "i1"), ("llen", "i1")])
GAPPED_DTYPE = np.dtype(
    [("seq1", "<i4"), ("pos1", "<i4"), ("seq2", "<i4"), ("pos2", "<i4"),
     ("score", "<i2"), ("ungapped", "<i2"), ("r_i", "<i2"), ("r_j", "<i2"),
     ("l_i", "<i2"), ("l_j", "<i2")])
ALIGN_DTYPE = np.dtype([(n, "<i4") for n in (
    "seq1", "seq2", "pos1", "pos2", "score", "q_start", "q_end", "s_start", "s_end", "length", "identities",
    "mismatches", "gap_opens")])
PLAST_XDROP = 38
ALIGN_BYTES = ALIGN_DTYPE.itemsize    # 52
HIT_BYTES = HIT_DTYPE.itemsize        # 20
GAPPED_BYTES = GAPPED_DTYPE.itemsize  # 28


PLAST_FILTER_S0 = 53  # the header's calibrated Section 4.2 filter threshold


class plast_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("w", "nl", "nr", "s1", "lg", "band", "gap_open", "gap_extend", "s2")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


COST_FIELDS = ("wide_slot", "wide_tile", "narrow_slot", "narrow_tile", "narrow4_slot", "narrow4_tile",
               "narrow2_slot", "narrow2_tile", "narrow16_slot", "narrow16_tile")


class plast_tile_costs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in COST_FIELDS[:8]] + \
        [("wide_int16_cells", ctypes.c_int32), ("wide_stage_depth", ctypes.c_int32)] + \
        [(n, ctypes.c_double) for n in COST_FIELDS[8:]]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class PlastError(RuntimeError):
    def __init__(self, call: str, code: int, needed: int | None = None):
        self.code = code
        self.needed = needed
        msg = f"{call}: {plast_strerror(code)} ({code})"
        if needed is not None:
            msg += f", needed {needed}"
        super().__init__(msg)


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libplast.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run paper_0804_3643_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        pI64 = ctypes.POINTER(ctypes.c_int64)
        pI32 = ctypes.POINTER(ctypes.c_int32)
        pPrm = ctypes.POINTER(plast_params)
        L.plast_default_params.argtypes = [pPrm]
        L.plast_default_params.restype = None
        L.plast_strerror.argtypes = [ctypes.c_int]
        L.plast_strerror.restype = ctypes.c_char_p
        L.plast_set_alloc_limit.argtypes = [i64]
        L.plast_set_alloc_limit.restype = ctypes.c_int
        L.plast_set_schedule.argtypes = [ctypes.c_int]
        L.plast_set_schedule.restype = ctypes.c_int
        L.plast_translate6.argtypes = [P, P, i32, P, i64, P, P, pI64, P]
        L.plast_translate6.restype = ctypes.c_int
        L.plast_index_bank.argtypes = [P, P, i32, pPrm, P, ctypes.POINTER(ctypes.c_void_p)]
        L.plast_index_bank.restype = ctypes.c_int
        L.plast_bank_free.argtypes = [P]
        L.plast_bank_free.restype = None
        L.plast_bank_stats.argtypes = [P, pI32, pI64, pI64]
        L.plast_bank_stats.restype = ctypes.c_int
        L.plast_bank_export_index.argtypes = [P, P, P, i64, pI64, P]
        L.plast_bank_export_index.restype = ctypes.c_int
        L.plast_ungapped.argtypes = [P, P, pPrm, P, i64, pI64, P]
        L.plast_ungapped.restype = ctypes.c_int
        L.plast_pair_count.argtypes = [P, P]
        L.plast_pair_count.restype = i64
        L.plast_small_gapped.argtypes = [P, P, pPrm, P, i64, P, i64, pI64, P]
        L.plast_small_gapped.restype = ctypes.c_int
        L.plast_search.argtypes = [P, P, pPrm, P, i64, pI64, P]
        L.plast_search.restype = ctypes.c_int
        L.plast_search_ex.argtypes = [P, P, pPrm, i32, P, i32, P, i64, pI64, pI64, P]
        L.plast_search_ex.restype = ctypes.c_int
        L.plast_ungapped_ex.argtypes = [P, P, pPrm, i32, P, i32, P, i64, pI64, P]
        L.plast_ungapped_ex.restype = ctypes.c_int
        L.plast_full_gapped.argtypes = [P, P, pPrm, i32, i32, P, i64, P, i64, pI64, pI64, P]
        L.plast_full_gapped.restype = ctypes.c_int
        L.plast_small_gapped_noalloc.argtypes = [P, P, pPrm, P, i64, P, i64, pI64, P]
        L.plast_small_gapped_noalloc.restype = ctypes.c_int
        L.plast_plan_create.argtypes = [P, P, pPrm, i32, i64, P, i64, P, ctypes.POINTER(ctypes.c_void_p)]
        L.plast_plan_create.restype = ctypes.c_int
        for f in ("plast_plan_run", "plast_plan_capture", "plast_plan_launch"):
            getattr(L, f).argtypes = [P, P]
            getattr(L, f).restype = ctypes.c_int
        L.plast_plan_result.argtypes = [P, pI64, pI64, P]
        L.plast_plan_result.restype = ctypes.c_int
        L.plast_plan_free.argtypes = [P]
        L.plast_plan_free.restype = None
        pCost = ctypes.POINTER(plast_tile_costs)
        L.plast_autotune.argtypes = [P, pCost]
        L.plast_autotune.restype = ctypes.c_int
        L.plast_get_tile_costs.argtypes = [pCost]
        L.plast_get_tile_costs.restype = ctypes.c_int
        L.plast_set_tile_costs.argtypes = [pCost]
        L.plast_set_tile_costs.restype = ctypes.c_int
        L.plast_stage2_tiles.argtypes = [P, P, i32, P, i64, pI64]
        L.plast_stage2_tiles.restype = ctypes.c_int
        L.plast_set_tile_shape.argtypes = [ctypes.c_int]
        L.plast_set_tile_shape.restype = ctypes.c_int
        L.plast_set_timing.argtypes = [ctypes.c_int]
        L.plast_set_timing.restype = ctypes.c_int
        L.plast_stage_times.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.plast_stage_times.restype = ctypes.c_int
        L.plast_kernel_launches.argtypes = []
        L.plast_kernel_launches.restype = ctypes.c_longlong
        L.plast_full_gapped_cells.argtypes = []
        L.plast_full_gapped_cells.restype = ctypes.c_int64
        _lib = L
    return _lib


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr() if t is not None and t.numel() else 0)


def _dev(t: torch.Tensor, dtype) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    return t.to(dtype).contiguous()


def plast_strerror(code: int) -> str:
    return lib().plast_strerror(code).decode()


def plast_default_params(**overrides) -> plast_params:
    p = plast_params()
    lib().plast_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, int(v))
    return p


def plast_set_alloc_limit(nbytes: int) -> None:
    """Fault injection: device allocations of the library above ``nbytes``
    fail with PLAST_E_OOM (0: no limit)."""
    rc = lib().plast_set_alloc_limit(int(nbytes))
    if rc:
        raise PlastError("plast_set_alloc_limit", rc)


def plast_set_schedule(mode: int) -> None:
    """0: one persistent launch with a device work queue; 1: one launch per key."""
    rc = lib().plast_set_schedule(int(mode))
    if rc:
        raise PlastError("plast_set_schedule", rc)


STAGES = ("upload_work_list", "stage2_kernel", "count_and_sort", "stage31_kernel", "threshold_and_write")


def plast_set_timing(on: bool) -> None:
    lib().plast_set_timing(1 if on else 0)


def plast_stage_times() -> dict:
    """Device ms of the stage intervals of this thread's last timed call."""
    ms = (ctypes.c_double * len(STAGES))()
    lib().plast_stage_times(ms, len(STAGES))
    return dict(zip(STAGES, list(ms)))


def plast_kernel_launches() -> int:
    return int(lib().plast_kernel_launches())


def plast_full_gapped_cells() -> int:
    """Dynamic-programming cells the last plast_full_gapped call of this
    thread computed (0 before any call and after a failed one)."""
    return int(lib().plast_full_gapped_cells())


def plast_autotune(stream=None) -> dict:
    c = plast_tile_costs()
    rc = lib().plast_autotune(_stream(stream), ctypes.byref(c))
    if rc:
        raise PlastError("plast_autotune", rc)
    return c.as_dict()


def plast_get_tile_costs() -> dict:
    c = plast_tile_costs()
    lib().plast_get_tile_costs(ctypes.byref(c))
    return c.as_dict()


def plast_set_tile_costs(costs: dict) -> None:
    c = plast_tile_costs(**{k: float(costs[k]) for k in COST_FIELDS},
                         wide_int16_cells=int(costs.get("wide_int16_cells", 12)),
                         wide_stage_depth=int(costs.get("wide_stage_depth", 1)))
    rc = lib().plast_set_tile_costs(ctypes.byref(c))
    if rc:
        raise PlastError("plast_set_tile_costs", rc)


def plast_set_tile_shape(mode: int) -> None:
    """0: by cost (default), 1: every tile wide, 2 / 3 / 4 / 5: every tile
    narrow of 8 / 4 / 2 / 16 rows."""
    rc = lib().plast_set_tile_shape(int(mode))
    if rc:
        raise PlastError("plast_set_tile_shape", rc)


def plast_stage2_tiles(key_off1: np.ndarray, key_off2: np.ndarray, n_sms: int = 0) -> np.ndarray:
    """Host-only: the stage-2 tiles [t, 6] = (key, first bank-1 CSR index,
    rows, shape, first and end bank-2 offset in the key's list) for two
    banks' CSR key offsets, long lists cut for a GPU of ``n_sms`` SMs."""
    k1 = np.ascontiguousarray(key_off1, dtype=np.int64)
    k2 = np.ascontiguousarray(key_off2, dtype=np.int64)
    if len(k1) != NKEYS + 1 or len(k2) != NKEYS + 1:
        raise ValueError("key offsets need NKEYS + 1 entries")
    n = ctypes.c_int64()
    cap = 0
    for _ in range(2):
        out = np.zeros((max(cap, 1), 6), dtype=np.int32)
        rc = lib().plast_stage2_tiles(k1.ctypes.data, k2.ctypes.data, int(n_sms), out.ctypes.data, cap,
                                      ctypes.byref(n))
        if rc == PLAST_E_CAPACITY:
            cap = n.value
            continue
        if rc:
            raise PlastError("plast_stage2_tiles", rc)
        return out[: n.value]
    raise PlastError("plast_stage2_tiles", PLAST_E_CAPACITY, n.value)


def _cost_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "plast_gb300", "tile_costs.json")


def autotune(cache: bool = True, stream=None) -> dict:
    """Tile costs of the current device: from the cache file when it holds an
    entry for this device and library build, else measured with
    plast_autotune (and stored).  Installs them and returns them."""
    import hashlib
    import json

    with open(LIB_PATH, "rb") as f:
        build_id = hashlib.sha256(f.read()).hexdigest()[:16]
    dev = torch.cuda.get_device_properties(torch.cuda.current_device())
    entry = f"{dev.name}|{dev.multi_processor_count}|{build_id}"
    path = _cost_cache_path()
    table = {}
    if cache and os.path.exists(path):
        try:
            with open(path) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
        if entry in table:
            plast_set_tile_costs(table[entry])
            return dict(table[entry], source="cache")
    costs = plast_autotune(stream)
    if cache:
        table[entry] = costs
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(table, f, indent=1)
        except OSError:
            pass
    return dict(costs, source="measured")


class Bank:
    """Owner of a plast_bank handle (freed with the object)."""

    def __init__(self, handle: ctypes.c_void_p):
        self.handle = handle
        n_seqs, n_res, n_idx = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        lib().plast_bank_stats(handle, ctypes.byref(n_seqs), ctypes.byref(n_res), ctypes.byref(n_idx))
        self.n_seqs, self.n_residues, self.n_positions = n_seqs.value, n_res.value, n_idx.value

    def free(self):
        if self.handle:
            lib().plast_bank_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def plast_index_bank(codes: torch.Tensor, seq_off: torch.Tensor, params: plast_params | None = None,
                     stream=None) -> Bank:
    codes = _dev(codes, torch.int8)
    seq_off = _dev(seq_off, torch.int64)
    h = ctypes.c_void_p()
    rc = lib().plast_index_bank(_ptr(codes), _ptr(seq_off), seq_off.numel() - 1,
                                ctypes.byref(params) if params is not None else None, _stream(stream),
                                ctypes.byref(h))
    if rc:
        raise PlastError("plast_index_bank", rc)
    return Bank(h)


def plast_bank_export_index(bank: Bank, stream=None):
    dev = torch.device("cuda", torch.cuda.current_device())
    key_off = torch.empty(NKEYS + 1, dtype=torch.int64, device=dev)
    pos = torch.empty(max(bank.n_positions, 1), dtype=torch.int32, device=dev)
    n = ctypes.c_int64()
    rc = lib().plast_bank_export_index(bank.handle, _ptr(key_off), _ptr(pos), pos.numel(), ctypes.byref(n),
                                       _stream(stream))
    if rc:
        raise PlastError("plast_bank_export_index", rc, n.value)
    return key_off, pos[:n.value]


def plast_pair_count(b1: Bank, b2: Bank) -> int:
    return int(lib().plast_pair_count(b1.handle, b2.handle))


def _records(out: torch.Tensor | None, cap: int, nbytes: int) -> torch.Tensor:
    if out is not None and out.numel() >= cap * nbytes:
        return out
    return torch.empty(max(cap, 1) * nbytes, dtype=torch.uint8, device=torch.device("cuda", torch.cuda.current_device()))


# The output count of the last automatically sized call of each kind on each
# pair of banks: a repeated call on the same banks is sized at once (the
# first guess from the pair count is run again with the exact count when it
# overflows, and banks with low-complexity runs overflow it).
_last_count: dict = {}


def _auto_cap(kind: str, b1: Bank, b2: Bank, guess: int) -> int:
    last = _last_count.get((kind, b1.handle.value, b2.handle.value))
    return max(guess, int(last * 1.05) + 4096) if last is not None else guess


def _note_count(kind: str, b1: Bank, b2: Bank, n: int) -> None:
    if len(_last_count) > 256:
        _last_count.clear()
    _last_count[(kind, b1.handle.value, b2.handle.value)] = n


def plast_ungapped(b1: Bank, b2: Bank, params: plast_params | None = None, cap: int | None = None,
                   out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Stage-2 hits as a uint8 device tensor [n, 20] (plast_hit records).
    With neither ``cap`` nor ``out`` given the output is sized automatically
    (one retry with the exact count); otherwise PLAST_E_CAPACITY raises."""
    auto = cap is None and out is None
    if cap is None:
        cap = (out.numel() // HIT_BYTES if out is not None
               else _auto_cap("ungapped", b1, b2, plast_pair_count(b1, b2) // 64 + 4096))
    for _ in range(2):
        buf = _records(out, cap, HIT_BYTES)
        n = ctypes.c_int64()
        rc = lib().plast_ungapped(b1.handle, b2.handle, ctypes.byref(params) if params is not None else None,
                                  _ptr(buf), cap, ctypes.byref(n), _stream(stream))
        if auto and rc in (0, PLAST_E_CAPACITY):
            _note_count("ungapped", b1, b2, n.value)
        if rc == PLAST_E_CAPACITY and auto:
            cap, out = n.value, None
            continue
        if rc:
            raise PlastError("plast_ungapped", rc, n.value)
        return buf[: n.value * HIT_BYTES].view(-1, HIT_BYTES)
    raise PlastError("plast_ungapped", PLAST_E_CAPACITY, cap)


def plast_small_gapped(b1: Bank, b2: Bank, hits: torch.Tensor, params: plast_params | None = None,
                       cap: int | None = None, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Stage-3.1 records (uint8 device tensor [n, 28]) of ``hits`` ([m, 20] plast_hit)."""
    hits = hits.contiguous()
    m = hits.numel() // HIT_BYTES
    if cap is None:
        cap = out.numel() // GAPPED_BYTES if out is not None else m
    buf = _records(out, cap, GAPPED_BYTES)
    n = ctypes.c_int64()
    rc = lib().plast_small_gapped(b1.handle, b2.handle, ctypes.byref(params) if params is not None else None,
                                  _ptr(hits), m, _ptr(buf), cap, ctypes.byref(n), _stream(stream))
    if rc:
        raise PlastError("plast_small_gapped", rc, n.value)
    return buf[: n.value * GAPPED_BYTES].view(-1, GAPPED_BYTES)


def plast_full_gapped(b1: Bank, b2: Bank, records: torch.Tensor, params: plast_params | None = None,
                      xdrop: int = PLAST_XDROP, s3: int = 47, cap: int | None = None, stream=None):
    """Stage 3.2 and the trace-back fields of stage-3.1 ``records`` ([m, 28]
    plast_gapped, device): (alignments [n, 52] uint8 device tensor of
    plast_alignment in canonical order, number of records extended)."""
    records = records.contiguous()
    m = records.numel() // GAPPED_BYTES
    cap = m if cap is None else cap
    buf = _records(None, cap, ALIGN_BYTES)
    n, ext = ctypes.c_int64(), ctypes.c_int64()
    rc = lib().plast_full_gapped(b1.handle, b2.handle, ctypes.byref(params) if params is not None else None,
                                 int(xdrop), int(s3), _ptr(records), m, _ptr(buf), cap, ctypes.byref(n),
                                 ctypes.byref(ext), _stream(stream))
    if rc:
        raise PlastError("plast_full_gapped", rc, n.value)
    return buf[: n.value * ALIGN_BYTES].view(-1, ALIGN_BYTES), ext.value


def alignments_numpy(t: torch.Tensor) -> np.ndarray:
    return t.contiguous().cpu().numpy().reshape(-1).view(ALIGN_DTYPE)


def alignments_tabular(al, names1=None, names2=None) -> list[str]:
    """Tab-separated lines of plast_alignment rows in the column order of
    BLAST's -m 8 report (the output Section 3.3.5 describes): query,
    subject, percent identity, alignment length, mismatches, gap opens,
    query start, query end, subject start, subject end (1-based, inclusive),
    then the raw score where -m 8 has the E-value and bit score, which need
    statistics the paper does not give.  ``al`` is a device tensor of records
    or their numpy view; names1 / names2 map sequence indices to names (the
    index itself by default)."""
    a = al if isinstance(al, np.ndarray) else alignments_numpy(al)
    out = []
    for r in a:
        q = names1[r["seq1"]] if names1 is not None else str(int(r["seq1"]))
        t = names2[r["seq2"]] if names2 is not None else str(int(r["seq2"]))
        length = int(r["length"])
        pid = 100.0 * int(r["identities"]) / length if length else 0.0
        out.append(f"{q}\t{t}\t{pid:.2f}\t{length}\t{int(r['mismatches'])}\t{int(r['gap_opens'])}\t"
                   f"{int(r['q_start']) + 1}\t{int(r['q_end'])}\t{int(r['s_start']) + 1}\t{int(r['s_end'])}\t"
                   f"{int(r['score'])}")
    return out


NOALLOC_MAX_HITS = 65536


def plast_small_gapped_noalloc(b1: Bank, b2: Bank, hits: torch.Tensor, out: torch.Tensor,
                               params: plast_params | None = None, stream=None) -> torch.Tensor:
    """plast_small_gapped for callers that cannot allocate: the library uses
    its fixed device scratch area (at most NOALLOC_MAX_HITS hits; calls that
    overlap on the GPU race).  ``out`` is the caller's preallocated uint8
    device buffer; the records are returned as a view of it."""
    hits = hits.contiguous()
    m = hits.numel() // HIT_BYTES
    cap = out.numel() // GAPPED_BYTES
    n = ctypes.c_int64()
    rc = lib().plast_small_gapped_noalloc(b1.handle, b2.handle,
                                          ctypes.byref(params) if params is not None else None,
                                          _ptr(hits), m, _ptr(out), cap, ctypes.byref(n), _stream(stream))
    if rc:
        raise PlastError("plast_small_gapped_noalloc", rc, n.value)
    return out[: n.value * GAPPED_BYTES].view(-1, GAPPED_BYTES)


def plast_search(b1: Bank, b2: Bank, params: plast_params | None = None, cap: int | None = None,
                 out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Stage-3.1 records [n, 28] (uint8 device tensor, canonical order);
    sized automatically unless ``cap`` or ``out`` is given, as plast_ungapped."""
    auto = cap is None and out is None
    if cap is None:
        cap = (out.numel() // GAPPED_BYTES if out is not None
               else _auto_cap("search", b1, b2, plast_pair_count(b1, b2) // 256 + 4096))
    for _ in range(2):
        buf = _records(out, cap, GAPPED_BYTES)
        n = ctypes.c_int64()
        rc = lib().plast_search(b1.handle, b2.handle, ctypes.byref(params) if params is not None else None,
                                _ptr(buf), cap, ctypes.byref(n), _stream(stream))
        if auto and rc in (0, PLAST_E_CAPACITY):
            _note_count("search", b1, b2, n.value)
        if rc == PLAST_E_CAPACITY and auto:
            cap, out = n.value, None
            continue
        if rc:
            raise PlastError("plast_search", rc, n.value)
        return buf[: n.value * GAPPED_BYTES].view(-1, GAPPED_BYTES)
    raise PlastError("plast_search", PLAST_E_CAPACITY, cap)


def _keys_arg(keys):
    """(host int32 array or None, ctypes pointer, count) of a key list (None = every key)."""
    if keys is None:
        return None, ctypes.c_void_p(0), 0
    k = np.ascontiguousarray(np.asarray(keys, dtype=np.int32))
    return k, k.ctypes.data_as(ctypes.c_void_p), len(k)


def plast_search_ex(b1: Bank, b2: Bank, params: plast_params | None = None, s0: int = 0, keys=None,
                    cap: int | None = None, out: torch.Tensor | None = None, stream=None):
    """plast_search with Section 4.2's filter threshold ``s0`` (0 = off) and
    an optional host list of subset-seed ``keys`` (None = every key):
    (records [n, 28] uint8 device tensor, number of stage-2 hits)."""
    auto = cap is None and out is None
    if cap is None:
        cap = (out.numel() // GAPPED_BYTES if out is not None
               else _auto_cap("search", b1, b2, plast_pair_count(b1, b2) // 256 + 4096))
    k, kp, nk = _keys_arg(keys)
    for _ in range(2):
        buf = _records(out, cap, GAPPED_BYTES)
        n, nu = ctypes.c_int64(), ctypes.c_int64()
        rc = lib().plast_search_ex(b1.handle, b2.handle, ctypes.byref(params) if params is not None else None,
                                   int(s0), kp, nk, _ptr(buf), cap, ctypes.byref(n), ctypes.byref(nu),
                                   _stream(stream))
        if auto and rc in (0, PLAST_E_CAPACITY) and keys is None and not s0:
            _note_count("search", b1, b2, n.value)
        if rc == PLAST_E_CAPACITY and auto:
            cap, out = n.value, None
            continue
        if rc:
            raise PlastError("plast_search_ex", rc, n.value)
        return buf[: n.value * GAPPED_BYTES].view(-1, GAPPED_BYTES), nu.value
    raise PlastError("plast_search_ex", PLAST_E_CAPACITY, cap)


class Plan:
    """plast_plan: a search of two banks with every buffer allocated up front
    (at most ``max_hits`` stage-2 hits, ``max_records`` records), runnable
    without allocation or host synchronisation and capturable in a CUDA
    graph.  The banks must outlive the plan."""

    def __init__(self, b1: Bank, b2: Bank, max_hits: int, max_records: int, params: plast_params | None = None,
                 s0: int = 0, stream=None):
        self.banks = (b1, b2)
        self.records = torch.empty(max(max_records, 1) * GAPPED_BYTES, dtype=torch.uint8,
                                   device=torch.device("cuda", torch.cuda.current_device()))
        self.handle = ctypes.c_void_p()
        rc = lib().plast_plan_create(b1.handle, b2.handle, ctypes.byref(params) if params is not None else None,
                                     int(s0), max_hits, _ptr(self.records), max_records, _stream(stream),
                                     ctypes.byref(self.handle))
        if rc:
            self.handle = None
            raise PlastError("plast_plan_create", rc)

    def _call(self, name, stream):
        rc = getattr(lib(), name)(self.handle, _stream(stream))
        if rc:
            raise PlastError(name, rc)

    def run(self, stream=None):
        self._call("plast_plan_run", stream)

    def capture(self, stream):
        self._call("plast_plan_capture", stream)

    def launch(self, stream=None):
        self._call("plast_plan_launch", stream)

    def result(self, stream=None):
        """(records [n, 28] uint8 view of the plan's output, stage-2 hits) of
        the last run; synchronises ``stream``."""
        n, nu = ctypes.c_int64(), ctypes.c_int64()
        rc = lib().plast_plan_result(self.handle, ctypes.byref(n), ctypes.byref(nu), _stream(stream))
        if rc:
            raise PlastError("plast_plan_result", rc, n.value)
        return self.records[: n.value * GAPPED_BYTES].view(-1, GAPPED_BYTES), nu.value

    def free(self):
        if self.handle:
            lib().plast_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def plast_ungapped_ex(b1: Bank, b2: Bank, params: plast_params | None = None, s0: int = 0, keys=None,
                      cap: int | None = None, stream=None) -> torch.Tensor:
    """plast_ungapped with Section 4.2's filter threshold ``s0`` (0 = off) and
    an optional host list of subset-seed ``keys`` (None = every key)."""
    k, kp, nk = _keys_arg(keys)
    if cap is None:
        cap = 1 << 20
    for _ in range(2):
        buf = _records(None, cap, HIT_BYTES)
        n = ctypes.c_int64()
        rc = lib().plast_ungapped_ex(b1.handle, b2.handle, ctypes.byref(params) if params is not None else None,
                                     int(s0), kp, nk, _ptr(buf), cap, ctypes.byref(n), _stream(stream))
        if rc == PLAST_E_CAPACITY:
            cap = n.value
            continue
        if rc:
            raise PlastError("plast_ungapped_ex", rc, n.value)
        return buf[: n.value * HIT_BYTES].view(-1, HIT_BYTES)
    raise PlastError("plast_ungapped_ex", PLAST_E_CAPACITY, cap)


def plast_translate6(dna: torch.Tensor, contig_off: torch.Tensor, stream=None):
    """(aa int8 [n], seq_off int64 [6c+1], meta int32 [6c, 2]) device tensors."""
    dna = _dev(dna, torch.uint8)
    contig_off = _dev(contig_off, torch.int64)
    c = contig_off.numel() - 1
    dev = dna.device
    aa = torch.empty(max(2 * dna.numel(), 1), dtype=torch.int8, device=dev)  # 6 frames x n/3 codons
    seq_off = torch.empty(6 * c + 1, dtype=torch.int64, device=dev)
    meta = torch.empty(max(12 * c, 1), dtype=torch.int32, device=dev)
    n = ctypes.c_int64()
    rc = lib().plast_translate6(_ptr(dna), _ptr(contig_off), c, _ptr(aa), aa.numel(), _ptr(seq_off), _ptr(meta),
                                ctypes.byref(n), _stream(stream))
    if rc:
        raise PlastError("plast_translate6", rc, n.value)
    return aa[: n.value], seq_off, meta[: 12 * c].view(-1, 2)


# ---------------------------------------------------------------------------
# Host-side views of the records (copies).
# ---------------------------------------------------------------------------
def hits_numpy(t: torch.Tensor) -> np.ndarray:
    return t.contiguous().cpu().numpy().reshape(-1).view(HIT_DTYPE)


def gapped_numpy(t: torch.Tensor) -> np.ndarray:
    return t.contiguous().cpu().numpy().reshape(-1).view(GAPPED_DTYPE)


def hits_from_numpy(a: np.ndarray, device=None) -> torch.Tensor:
    a = np.ascontiguousarray(a, dtype=HIT_DTYPE)
    t = torch.from_numpy(a.view(np.uint8).reshape(-1, HIT_BYTES).copy())
    return t.to(device or torch.device("cuda", torch.cuda.current_device()))


@dataclass
class DeviceBank:
    """A bank's codes and offsets on the device, as plast_index_bank takes them."""
    codes: torch.Tensor
    seq_off: torch.Tensor

    @staticmethod
    def from_host(codes: np.ndarray, seq_off: np.ndarray, device=None) -> "DeviceBank":
        dev = device or torch.device("cuda", torch.cuda.current_device())
        return DeviceBank(torch.from_numpy(np.ascontiguousarray(codes).view(np.int8)).to(dev),
                          torch.from_numpy(np.ascontiguousarray(seq_off, dtype=np.int64)).to(dev))
