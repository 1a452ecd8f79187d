#!/usr/bin/env python
"""Benchmark of the hot path: one step = stage 0 indexing of both banks,
stages 1-2 (ungapped extension of every pair of every shared key), stage
3.1 (small gapped extension of the survivors) and the sort of the passing
records, on the 10,000 x 100,000 synthetic protein workload, through the C
ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``value`` is ungapped pairs per second of the
whole step with the banks' codes resident in device memory; ``e2e`` is the
same metric with the codes copied from pinned host memory and the records
copied back inside the timed region.  ``roofline`` rates the dominant kernel
(stage 2) against the integer ALU peak; ``cpu_baseline`` times the CPU oracle
on a bounded sample of the same workload.  ``--impl reference`` times the CPU
oracle alone (the reference arm of this comparison).

Multi-GPU (torchrun): every rank compares the shared bank 1 with its own
bank-2 shard (weak scaling); no collective touches the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0804_3643_gb300 import synth  # noqa: E402

WORKLOAD = "plastp_full"
CELLS_PER_PAIR = 48        # ungapped window: 26 right + 22 left cells
CELLS_PER_CLK_SM = 128     # int16 cells per clock per SM on the ALU / FMA-heavy pipes
BAND_CELLS_PER_HIT = 2 * 64 * 17  # stage 3.1: two sides x LG rows x (2 x band + 1) columns
ALU_LANES_PER_CLK_SM = 64  # ALU-pipe lanes per clock per SM (every integer max issues there)
METRIC = "ungapped pairs/s and GCUPS at 1 GB300 (bit-exact), % of int/HBM roofline"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# --------------------------------------------------------------------------
# nvidia-smi clock sampler (runs during the timed region)
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path:
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        smax = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [x for x in sm if x >= 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("[N/A]",))}


# --------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline and the reference arm)
# --------------------------------------------------------------------------
def oracle_sample_keys(o1, o2, target_pairs: float, seed: int = 7):
    n1 = np.diff(o1.idx.key_off)
    n2 = np.diff(o2.idx.key_off)
    order = np.random.default_rng(seed).permutation(len(n1))
    keys, pairs = [], 0
    for k in order:
        p = int(n1[k] * n2[k])
        if p == 0:
            continue
        keys.append(int(k))
        pairs += p
        if pairs >= target_pairs:
            break
    return sorted(keys), pairs


def oracle_step(oracle, o1, o2, keys, threads, prm):
    """Stages 1-2 over the sampled keys, then stage 3.1 of their hits."""
    h = oracle.ungapped(o1, o2, prm, keys=keys, threads=threads)
    oracle.small_gapped(o1, o2, h, prm, threads=threads)
    return len(h)


# One fixed sample of keys for both CPU arms (the cpu_baseline leg and the
# --impl reference line): the keys drawn with this seed until they hold
# this many pairs, so the two arms time the same work.
SAMPLE_SEED = 7
SAMPLE_PAIRS = 1.2e8


def run_oracle(b1, b2, steps: int, warmup: int, threads: int | None = None, s0: int = 0):
    import oracle

    prm = oracle.Params(s0=s0)
    threads = threads or os.cpu_count() or 1
    t0 = time.time()
    o1 = oracle.make_bank(b1.codes, b1.seq_off)
    o2 = oracle.make_bank(b2.codes, b2.seq_off)
    t_index = time.time() - t0
    keys, pairs = oracle_sample_keys(o1, o2, SAMPLE_PAIRS, seed=SAMPLE_SEED)
    for _ in range(warmup):
        oracle_step(oracle, o1, o2, keys, threads, prm)
    times = []
    for _ in range(steps):
        t0 = time.time()
        oracle_step(oracle, o1, o2, keys, threads, prm)
        times.append(time.time() - t0)
    per = sum(times) / len(times)
    total_pairs = float((np.diff(o1.idx.key_off) * np.diff(o2.idx.key_off)).sum())
    return {
        "value": pairs / per, "unit": "pairs/s", "cores": threads, "kind": "oracle",
        "sample": f"{len(keys)} of 8800 keys drawn at random (seed {SAMPLE_SEED}, until {SAMPLE_PAIRS:.2g} pairs: "
                  f"{pairs:.4e} of {total_pairs:.4e} pairs): stages 1-2 and 3.1 of those keys per step, "
                  f"{steps} timed steps, plain C -O2 with {threads} threads; stage-0 indexing of the full "
                  f"banks took {t_index:.2f} s once, outside the timed steps",
        "seconds_per_step": per, "total_pairs": int(total_pairs),
    }


def headline_config(b1, b2, pairs: int, scale: float, bank2_proteins, s0: int, world: int) -> dict:
    """The workload the metric is quoted on (the same dict in both arms' lines)."""
    full = scale == 1.0 and not bank2_proteins
    d = {
        "workload": f"PLAST-P {'full scale' if full else 'reduced'}: {b1.n_seqs} x {b2.n_seqs} synthetic proteins "
                    f"({len(b1.codes)} / {len(b2.codes)} residues), 5% planted homologs, seed 1",
        "step": "index both banks + ungapped all pairs + small gapped + sort of the records"
                + (f" (Section 4.2 filter on, S0 = {s0}: lossy, fewer hits)" if s0 else ""),
        "pairs_per_step": int(pairs),
        "params": {"w": 4, "nl": 22, "nr": 22, "s1": 38, "lg": 64, "band": 8, "gap_open": 11, "gap_extend": 1,
                   "s2": 47, "s0": s0},
        "l2": "inputs larger than L2 (129 MB): 1.7 GB of neighbourhood arrays rebuilt and read every step, "
              "no explicit flush",
        "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
    }
    return d


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def reduce_max(x: float, world: int, device) -> float:
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling:
    every rank processes the same amount)."""
    return world * units_per_rank / (ms_max / 1e3)


def shard_seed(rank: int) -> int:
    """Seed of a rank's bank-2 shard: rank 0 draws the single-GPU workload."""
    return 1 + rank


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("ungapped.cu", "ungapped.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_0804_3643_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic():
    """Per-launch DRAM traffic of the stage-2 kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    try:
        with open(os.path.join(ROOT, "profiles", "ungapped_traffic.json")) as f:
            t = json.load(f)
    except OSError:
        return None
    if t.get("kernel_source_hash") != kernel_source_hash():
        return None
    return t


def stage31_roofline(hits: int, ms: float, n_sm: int, sm_max: float, sm_mhz) -> dict:
    """Stage 3.1 against the integer ALU peak.  Unit: one band cell of the
    small gapped extension (2 sides x 64 rows x 17 columns per stage-2
    survivor, the cells off the grid included).  Per cell the affine
    recurrence takes its maxima on the ALU pipe, two cells (two hits) per
    int16x2 instruction; the peak counts three fused add-max instructions per
    cell pair (the E, F and H updates), 64 lanes x 2 / 3 = 42.7 cells per clock
    per SM.  The kernel issues four per cell pair, the fewest this instruction
    set allows (H takes the maximum of three terms one of which needs an add of
    a table value), so `frac_of_4op_floor` rates it against 32 cells per clock
    per SM as well."""
    cells = hits * BAND_CELLS_PER_HIT
    achieved = cells / (ms / 1e3)
    per_clk = ALU_LANES_PER_CLK_SM * 2 / 3
    peak = n_sm * per_clk * sm_max * 1e6
    floor4 = n_sm * ALU_LANES_PER_CLK_SM * 2 / 4 * sm_max * 1e6
    return {
        "bound": "alu",
        "kernel": "stage 3.1: k_small_gapped (every stage-2 survivor: both sides' scores and end cells)",
        "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tcell/s", "frac": achieved / peak,
        "traffic": None, "cells_per_hit": BAND_CELLS_PER_HIT, "kernel_ms": ms,
        "peak_basis": f"{n_sm} SMs x {per_clk:.2f} cells/clock (ALU pipe 64 lanes x 2 int16 halves / 3 fused "
                      f"add-max per cell) x {sm_max:.0f} MHz (max SM clock)",
        "frac_of_4op_floor": achieved / floor4,
        "frac_at_measured_clock": achieved / (n_sm * per_clk * sm_mhz * 1e6) if sm_mhz else None,
    }


def setup_tiles(args, B) -> dict:
    """Stage-2 tile shape policy and its cost constants (measured on this
    device by the library's calibration unless --no-autotune)."""
    B.plast_set_tile_shape({"auto": 0, "wide": 1, "narrow": 2, "narrow4": 3, "narrow2": 4, "narrow16": 5}[args.tile_shape])
    if args.no_autotune:
        c = dict(B.plast_get_tile_costs(), source="defaults")
    else:
        t0 = time.time()
        c = B.autotune()
        log(f"tile costs ({c['source']}, {time.time() - t0:.2f}s): {c}")
    if args.wide_int16_cells is not None:
        B.plast_set_tile_costs(dict(c, wide_int16_cells=args.wide_int16_cells))
        c = dict(c, wide_int16_cells=args.wide_int16_cells, source=c["source"] + ", variant forced")
    return dict(c, shape=args.tile_shape)


def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_0804_3643_gb300 import binding as B
    from paper_0804_3643_gb300 import build

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if not os.path.exists(build.LIB):
        build.build()
    B.lib()
    B.plast_set_schedule(1 if args.schedule == "per_key" else 0)
    tiles = setup_tiles(args, B)
    prm = B.plast_default_params()

    t0 = time.time()
    b1, _ = synth.workload(WORKLOAD, seed=1, scale=args.scale, n2=2)
    # weak scaling: each rank its own bank-2 shard of the same size
    _, b2 = synth.workload(WORKLOAD, seed=shard_seed(rank), scale=args.scale, n2=args.bank2_proteins)
    log(f"[rank {rank}] banks generated in {time.time() - t0:.1f}s: {b1.n_seqs} x {b2.n_seqs} proteins, "
        f"{len(b1.codes)} / {len(b2.codes)} residues")

    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    h1c, h1o = pin(b1.codes.view(np.int8)), pin(b1.seq_off)
    h2c, h2o = pin(b2.codes.view(np.int8)), pin(b2.seq_off)
    d1c, d1o = h1c.to(dev), h1o.to(dev)
    d2c, d2o = h2c.to(dev), h2o.to(dev)
    stream = torch.cuda.current_stream()

    # size the output once
    g1 = B.plast_index_bank(d1c, d1o)
    g2 = B.plast_index_bank(d2c, d2o)
    pairs = B.plast_pair_count(g1, g2)
    recs, n_ung = B.plast_search_ex(g1, g2, prm, s0=args.s0)
    cap = int(recs.shape[0] * 1.05) + 1024
    out = torch.empty(cap * B.GAPPED_BYTES, dtype=torch.uint8, device=dev)
    n_recs = recs.shape[0]
    del recs
    nb_gb = (g1.n_positions + g2.n_positions) * CELLS_PER_PAIR / 1e9
    g1.free()
    g2.free()
    torch.cuda.synchronize()
    log(f"[rank {rank}] pairs/step {pairs:.4e}, stage-2 hits {n_ung}, records {n_recs}")

    stage_ms = []

    def step(c1, o1_, c2, o2_):
        a = B.plast_index_bank(c1, o1_)
        b = B.plast_index_bank(c2, o2_)
        if args.s0:
            r, _ = B.plast_search_ex(a, b, prm, s0=args.s0, out=out, cap=cap)
        else:
            r = B.plast_search(a, b, prm, out=out, cap=cap)
        stage_ms.append(B.plast_stage_times())
        a.free()
        b.free()
        return r

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x):
        return reduce_max(x, world, dev)

    # ---- device-resident arm
    B.plast_set_timing(True)
    for _ in range(args.warmup):
        step(d1c, d1o, d2c, d2o)
    stage_ms.clear()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        launches0 = B.plast_kernel_launches()
        e0.record(stream)
        for _ in range(args.steps):
            step(d1c, d1o, d2c, d2o)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = B.plast_kernel_launches() - launches0
        barrier()
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    clocks = clk.summary()
    ung_ms = statistics.mean(s["stage2_kernel"] for s in stage_ms)
    gap_ms = statistics.mean(s["stage31_kernel"] for s in stage_ms)
    stages = {name: round(statistics.mean(s[name] for s in stage_ms), 3) for name in B.STAGES}

    # ---- end-to-end arm: host buffers in, records out
    rec_bytes = n_recs * B.GAPPED_BYTES
    host_out = torch.empty(max(rec_bytes, 1), dtype=torch.uint8).pin_memory()

    def e2e_step():
        c1, o1_ = h1c.to(dev, non_blocking=True), h1o.to(dev, non_blocking=True)
        c2, o2_ = h2c.to(dev, non_blocking=True), h2o.to(dev, non_blocking=True)
        r = step(c1, o1_, c2, o2_)
        host_out[: r.numel()].copy_(r.reshape(-1), non_blocking=True)

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    B.plast_set_timing(False)
    h2d = int(h1c.numel() + h1o.numel() * 8 + h2c.numel() + h2o.numel() * 8)

    pk = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    # A cell needs one int16 max (ALU pipe: 64 lanes x 2 halves per clock per
    # SM) and one int16 add (FMA-heavy pipe, the same rate): 128 cells per
    # clock per SM.  The pipe of each instruction and the issue rates are the
    # ones the probe in paper_0804_3643_gb300/probe/pipes.cu measures.
    peak_cells = n_sm * CELLS_PER_CLK_SM * sm_max * 1e6
    achieved_cells = pairs * CELLS_PER_PAIR / (ung_ms / 1e3)
    tr = committed_traffic()
    traffic = None
    if tr is not None:
        traffic = tr["dram_bytes_per_pair"] * pairs
    result = {
        "metric": METRIC,
        "value": whole_job_rate(pairs, world, ms_step),
        "unit": "pairs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int16",
        "data": "synthetic",
        "config": headline_config(b1, b2, pairs, args.scale, args.bank2_proteins, args.s0, world),
        "run": {
            "stage2_hits_per_step": n_ung,
            "records_per_step": n_recs,
            "schedule": args.schedule,
            "stage2_tiles": tiles,
            "neighbourhood_gb": round(nb_gb, 3),
        },
        "gcups": world * pairs * CELLS_PER_PAIR / (ms_step / 1e3) / 1e9,
        "stage_ms": stages,
        "roofline": {
            "bound": "alu",
            "kernel": f"stage 2: k_ungapped<{tiles.get('wide_int16_cells', '?')}> (wide tiles) then "
                      "k_ungapped_narrow (narrow tiles), timed together",
            "achieved": achieved_cells / 1e12,
            "peak": peak_cells / 1e12,
            "unit": "Tcell/s",
            "frac": achieved_cells / peak_cells,
            "traffic": traffic,
            "cells_per_pair": CELLS_PER_PAIR,
            "kernel_ms": ung_ms,
            "peak_basis": f"{n_sm} SMs x {CELLS_PER_CLK_SM} cells/clock (ALU pipe 64 lanes x 2 int16 halves for "
                          f"the max, FMA-heavy pipe the same for the add) x {sm_max:.0f} MHz (max SM clock)",
            "frac_at_measured_clock": (achieved_cells / (n_sm * CELLS_PER_CLK_SM * clocks["sm_mhz"] * 1e6)
                                       if clocks.get("sm_mhz") else None),
            "hbm_gbs": (traffic / (ung_ms / 1e3) / 1e9) if traffic else None,
        },
        "roofline_stage31": stage31_roofline(n_ung, gap_ms, n_sm, sm_max, clocks.get("sm_mhz")),
        "e2e": {"value": world * pairs / (e2e_ms / 1e3), "unit": "pairs/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": int(rec_bytes), "ms_per_step": e2e_ms},
        "clocks": clocks,
        "gpu_launches": int(launches),
        "gpu_launches_per_step": launches / args.steps,
    }
    return result, (b1, b2)

# --------------------------------------------------------------------------
# Other workloads (not the headline line): the batching stress test, the
# TPLAST-N chain and the serving loop.  Each prints one JSON line.
# --------------------------------------------------------------------------
def _time_steps(fn, steps, warmup):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_stress(args, steps=None, warmup=None, tiles=None):
    """50,000 x 50,000 proteins, 20 % with low-complexity runs: heavy-tailed
    key lists; the persistent work-queue launch against one launch per key."""
    import torch

    from paper_0804_3643_gb300 import binding as B

    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    tiles = setup_tiles(args, B) if tiles is None else tiles
    b1, b2 = synth.workload("batching_stress", seed=1, scale=args.scale)
    d1 = B.DeviceBank.from_host(b1.codes, b1.seq_off)
    d2 = B.DeviceBank.from_host(b2.codes, b2.seq_off)
    g1 = B.plast_index_bank(d1.codes, d1.seq_off)
    g2 = B.plast_index_bank(d2.codes, d2.seq_off)
    pairs = B.plast_pair_count(g1, g2)
    recs, n_ung = B.plast_search_ex(g1, g2)
    cap = int(recs.shape[0] * 1.05) + 1024
    out = torch.empty(cap * B.GAPPED_BYTES, dtype=torch.uint8, device="cuda")
    res = {}
    B.plast_set_timing(True)
    for name, mode in (("persistent", 0), ("per_key", 1)):
        B.plast_set_schedule(mode)
        st = []

        def step():
            B.plast_search(g1, g2, out=out, cap=cap)
            st.append(B.plast_stage_times())

        ms = _time_steps(step, steps, warmup)
        res[name] = {"ms_per_search": ms, "pairs_per_s": pairs / (ms / 1e3),
                     "stage2_ms": statistics.mean(x["stage2_kernel"] for x in st[warmup:])}
    B.plast_set_schedule(0)
    B.plast_set_timing(False)
    n1 = np.diff(np.array(B.plast_bank_export_index(g1)[0].cpu()))
    n2 = np.diff(np.array(B.plast_bank_export_index(g2)[0].cpu()))
    per_key = n1 * n2
    return {
        "metric": "search time, persistent work queue vs one launch per key", "unit": "ms",
        "workload": f"batching stress: {b1.n_seqs} x {b2.n_seqs} proteins, 20% with low-complexity runs, seed 1",
        "pairs": pairs, "stage2_hits": n_ung, "records": int(recs.shape[0]),
        "pairs_per_key": {"max": int(per_key.max()), "p50": float(np.median(per_key[per_key > 0])),
                          "keys_over_1e6": int((per_key > 1e6).sum())},
        "schedules": res, "stage2_tiles": tiles,
        "speedup_persistent_over_per_key": res["per_key"]["ms_per_search"] / res["persistent"]["ms_per_search"],
    }


def run_tplastn(args):
    """5,000 proteins vs a 50 Mbp nucleotide bank: six-frame translation on
    the device, then stage 0 of both banks and the search, per step."""
    import torch

    from paper_0804_3643_gb300 import binding as B

    tiles = setup_tiles(args, B)
    b1, dna = synth.tplastn_workload(seed=1, scale=args.scale)
    d1 = B.DeviceBank.from_host(b1.codes, b1.seq_off)
    hd = torch.from_numpy(dna.codes).cuda()
    ho = torch.from_numpy(dna.seq_off).cuda()
    aa, so, _ = B.plast_translate6(hd, ho)
    g1 = B.plast_index_bank(d1.codes, d1.seq_off)
    g2 = B.plast_index_bank(aa, so)
    pairs = B.plast_pair_count(g1, g2)
    recs, n_ung = B.plast_search_ex(g1, g2)
    cap = int(recs.shape[0] * 1.05) + 1024
    out = torch.empty(cap * B.GAPPED_BYTES, dtype=torch.uint8, device="cuda")
    n_rec = int(recs.shape[0])
    del g2

    def step():
        a, s_, _ = B.plast_translate6(hd, ho)
        x = B.plast_index_bank(d1.codes, d1.seq_off)
        y = B.plast_index_bank(a, s_)
        B.plast_search(x, y, out=out, cap=cap)
        x.free()
        y.free()

    ms = _time_steps(step, args.steps, args.warmup)
    return {
        "metric": "ungapped pairs/s, TPLAST-N chain (translate6 + index + search)", "unit": "pairs/s",
        "value": pairs / (ms / 1e3), "ms_per_step": ms,
        "workload": f"TPLAST-N: {b1.n_seqs} proteins vs {len(dna.codes) / 1e6:.1f} Mbp in {dna.n_seqs} contigs "
                    f"({len(aa)} translated residues), {len(dna.planted['regions'])} planted regions, seed 1",
        "pairs": pairs, "stage2_hits": n_ung, "records": n_rec, "stage2_tiles": tiles,
    }


def run_plastx(args):
    """PLAST-X: 1,000 nucleotide sequences of about 1 kbp vs a 50 Mbp
    nucleotide bank, both translated in six frames on the device, then
    stage 0 of both translated banks and the search, per step."""
    import torch

    from paper_0804_3643_gb300 import binding as B

    tiles = setup_tiles(args, B)
    q, subj = synth.plastx_workload(seed=1, scale=args.scale)
    hq, oq = torch.from_numpy(q.codes).cuda(), torch.from_numpy(q.seq_off).cuda()
    hs, os_ = torch.from_numpy(subj.codes).cuda(), torch.from_numpy(subj.seq_off).cuda()
    a1, s1, _ = B.plast_translate6(hq, oq)
    a2, s2, _ = B.plast_translate6(hs, os_)
    g1 = B.plast_index_bank(a1, s1)
    g2 = B.plast_index_bank(a2, s2)
    pairs = B.plast_pair_count(g1, g2)
    recs, n_ung = B.plast_search_ex(g1, g2)
    cap = int(recs.shape[0] * 1.05) + 1024
    out = torch.empty(cap * B.GAPPED_BYTES, dtype=torch.uint8, device="cuda")
    n_rec = int(recs.shape[0])
    n_aa = (len(a1), len(a2))
    del g1, g2, a1, a2, s1, s2

    def step():
        x_aa, x_so, _ = B.plast_translate6(hq, oq)
        y_aa, y_so, _ = B.plast_translate6(hs, os_)
        x = B.plast_index_bank(x_aa, x_so)
        y = B.plast_index_bank(y_aa, y_so)
        B.plast_search(x, y, out=out, cap=cap)
        x.free()
        y.free()

    ms = _time_steps(step, args.steps, args.warmup)
    return {
        "metric": "ungapped pairs/s, PLAST-X chain (translate6 of both banks + index + search)", "unit": "pairs/s",
        "value": pairs / (ms / 1e3), "ms_per_step": ms,
        "workload": f"PLAST-X: {q.n_seqs} sequences ({len(q.codes) / 1e6:.2f} Mbp) vs {len(subj.codes) / 1e6:.1f} Mbp "
                    f"in {subj.n_seqs} sequences ({n_aa[0]} / {n_aa[1]} translated residues), "
                    f"{len(q.planted['regions'])} / {len(subj.planted['regions'])} planted regions, seed 1",
        "pairs": pairs, "stage2_hits": n_ung, "records": n_rec, "stage2_tiles": tiles,
    }


def run_query(args, steps=None, warmup=None, tiles=None):
    """One query bank of --query-proteins proteins against a resident bank of
    --bank2-proteins (default 1,000,000): the search a serving request runs,
    timed three ways: the plain call (plast_search: work list, allocation and
    the survivor-count read on the host), the planned search (buffers
    allocated once, no host synchronisation inside) and its CUDA-graph
    replay."""
    import torch

    from paper_0804_3643_gb300 import binding as B

    B.lib()
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    tiles = setup_tiles(args, B) if tiles is None else tiles
    n_bank = args.bank2_proteins or 1_000_000
    t0 = time.time()
    bank = synth.random_protein_bank(np.random.default_rng(1), max(2, int(n_bank * args.scale)))
    q = synth.random_protein_bank(np.random.default_rng(2), args.query_proteins)
    db = B.DeviceBank.from_host(bank.codes, bank.seq_off)
    dq = B.DeviceBank.from_host(q.codes, q.seq_off)
    gb = B.plast_index_bank(db.codes, db.seq_off)
    gq = B.plast_index_bank(dq.codes, dq.seq_off)
    log(f"banks ready in {time.time() - t0:.1f}s")
    pairs = B.plast_pair_count(gq, gb)
    ref, n_ung = B.plast_search_ex(gq, gb)
    st = torch.cuda.Stream()
    plan = B.Plan(gq, gb, max_hits=2 * n_ung + 4096, max_records=2 * ref.shape[0] + 1024, stream=st)
    plan.capture(st)
    res = {}
    with torch.cuda.stream(st):
        res["search_ms"] = _time_steps(lambda: B.plast_search(gq, gb, stream=st), steps, warmup)
        res["plan_ms"] = _time_steps(lambda: (plan.run(st), plan.result(st)), steps, warmup)
        res["graph_ms"] = _time_steps(lambda: (plan.launch(st), plan.result(st)), steps, warmup)
    recs, nu = plan.result(st)
    if not (torch.equal(recs, ref) and nu == n_ung):
        raise RuntimeError("planned search differs from plast_search")
    B.plast_set_timing(True)
    stages = []
    for _ in range(3):
        B.plast_search(gq, gb, stream=st)
        stages.append(B.plast_stage_times())
    B.plast_set_timing(False)
    res["stage_ms"] = {k: round(statistics.median(x[k] for x in stages), 3) for k in stages[0]}
    t1 = time.perf_counter()
    gq2 = B.plast_index_bank(dq.codes, dq.seq_off, stream=st)
    st.synchronize()
    res["query_index_ms"] = (time.perf_counter() - t1) * 1e3
    del gq2
    # rebuilding the resident bank's index from its codes (already on the
    # device): the alternative to keeping a serialised index on disk, whose
    # windows alone take 48 bytes per residue
    del plan, gb
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    gb = B.plast_index_bank(db.codes, db.seq_off, stream=st)
    st.synchronize()
    res["resident_index_ms"] = (time.perf_counter() - t1) * 1e3
    res["resident_windows_gb"] = round(48 * len(bank.codes) / 1e9, 2)
    return {
        "metric": "query search latency against a resident bank (plain call / planned / CUDA graph)", "unit": "ms",
        "workload": f"{q.n_seqs} random proteins ({len(q.codes)} residues) vs a resident bank of {bank.n_seqs} "
                    f"random proteins ({len(bank.codes)} residues)",
        "pairs": pairs, "stage2_hits": n_ung, "records": int(ref.shape[0]),
        **res, "pairs_per_s_graph": pairs / (res["graph_ms"] / 1e3), "stage2_tiles": tiles,
    }


def run_serving(args, rates=(5.0, 20.0, 50.0, 100.0, 200.0), tiles=None):
    """A resident bank of 1,000,000 proteins; query banks of 1-500 proteins
    arriving as Poisson processes at each of `rates` per second; continuous
    batching."""
    from paper_0804_3643_gb300 import binding as B
    from paper_0804_3643_gb300 import serve

    B.lib()
    tiles = setup_tiles(args, B) if tiles is None else tiles
    rng = np.random.default_rng(1)
    n_res = max(1000, int(1_000_000 * args.scale))
    t0 = time.time()
    bank = synth.random_protein_bank(rng, n_res)
    ex = serve.GpuExecutor(bank.codes, bank.seq_off)
    log(f"resident bank {n_res} proteins ({len(bank.codes)} residues) generated and indexed in "
        f"{time.time() - t0:.1f}s")
    rows = []
    for rate in rates:
        reqs = [serve.Request(i, t, b.codes, b.seq_off) for i, (t, b) in
                enumerate(synth.serving_requests(seed=int(rate), n=args.requests, rate_per_s=rate))]
        srv = serve.Server(ex.execute, ex.mem_of, slots=2, mem_budget=120 << 30, max_batch_seqs=3000)
        t1 = time.perf_counter()
        srv.run(reqs, realtime=True, timeout=900)
        wall = time.perf_counter() - t1
        pairs = sum(b.pairs for b in srv.batches)
        row = {"rate_per_s": rate, **serve.latency_summary(reqs, pairs, wall),
               "batches": len(srv.batches), "mean_batch_requests": len(reqs) / len(srv.batches),
               "peak_concurrent_batches": srv.peak_busy, "wall_s": wall}
        log(json.dumps(row))
        rows.append(row)
    return {"metric": "serving latency p50/p99 and pairs/s under continuous batching", "unit": "ms",
            "workload": f"resident bank of {n_res} synthetic proteins ({len(bank.codes)} residues); "
                        f"{args.requests} query banks of U(1..500) proteins per rate, Poisson arrivals",
            "slots": 2, "stage2_tiles": tiles, "rows": rows}



def run_stage32(args, steps: int = 3) -> dict:
    """Stage 3.2 (full gapped extension with the drop-off, trace-back fields,
    redundancy lists) of the stage-3.1 records of the full-scale search,
    through plast_full_gapped: the kernel time from the library's stage
    events and the whole call (ordering, kernel, compaction)."""
    import torch

    from paper_0804_3643_gb300 import binding as B

    B.lib()
    b1, _ = synth.workload(WORKLOAD, seed=1, scale=args.scale, n2=2)
    _, b2 = synth.workload(WORKLOAD, seed=1, scale=args.scale, n2=args.bank2_proteins)
    d1 = B.DeviceBank.from_host(b1.codes, b1.seq_off)
    d2 = B.DeviceBank.from_host(b2.codes, b2.seq_off)
    g1 = B.plast_index_bank(d1.codes, d1.seq_off)
    g2 = B.plast_index_bank(d2.codes, d2.seq_off)
    recs, _ = B.plast_search_ex(g1, g2)
    B.plast_full_gapped(g1, g2, recs)  # warm-up
    B.plast_set_timing(True)
    kern, call = [], []
    for _ in range(steps):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        al, ext = B.plast_full_gapped(g1, g2, recs)
        torch.cuda.synchronize()
        call.append((time.perf_counter() - t1) * 1e3)
        kern.append(B.plast_stage_times()["upload_work_list"])  # interval 0: the extension kernel
    B.plast_set_timing(False)
    cells = B.plast_full_gapped_cells()
    k_ms = statistics.median(kern)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    sm_max = float(peaks().get("sm_max_mhz", 2070.0))
    peak = n_sm * ALU_LANES_PER_CLK_SM * 2 / 3 * sm_max * 1e6
    return {
        "metric": "stage 3.2 (full gapped extension, trace-back fields) of a search's stage-3.1 records",
        "unit": "ms",
        "workload": f"the {recs.shape[0]} stage-3.1 records of the search of {b1.n_seqs} x {b2.n_seqs} synthetic "
                    f"proteins (seed 1)",
        "records": int(recs.shape[0]), "extended": int(ext), "alignments": int(al.shape[0]),
        "xdrop": B.PLAST_XDROP, "kernel_ms": round(k_ms, 3), "call_ms": round(statistics.median(call), 3),
        "records_per_s": recs.shape[0] / (k_ms / 1e3),
        "cells": cells, "gcups": cells / (k_ms / 1e3) / 1e9,
        "roofline": {
            "bound": "alu", "kernel": "k_full_gapped", "unit": "Tcell/s",
            "achieved": cells / (k_ms / 1e3) / 1e12, "peak": peak / 1e12,
            "frac": cells / (k_ms / 1e3) / peak,
            "peak_basis": f"{n_sm} SMs x {ALU_LANES_PER_CLK_SM * 2 / 3:.2f} cells/clock (three fused add-max "
                          f"instructions per cell, two cells per int16x2 instruction, as for stage 3.1) x "
                          f"{sm_max:.0f} MHz; unit: every computed cell of every extended side, dropped ones "
                          f"included (plast_full_gapped_cells)",
        },
        "timing": f"kernel: CUDA events on the call's stream, median of {steps}; call: host wall time",
    }


def run_extras(args, tiles) -> dict:
    """Secondary targets measured after the headline (not part of its timed
    region): the batching-stress workload (50,000 x 50,000 proteins with
    low-complexity runs) under the persistent work queue and under one launch
    per key, stage 3.2 on the headline search's records, one 250-protein
    query against a resident 1,000,000-protein bank as a plain call, a
    planned search and its CUDA-graph replay, and the serving loop at 20
    requests per second."""
    import torch

    out = {}
    t0 = time.time()
    s = run_stress(args, steps=2, warmup=1, tiles=tiles)
    out["batching_stress"] = {
        "workload": s["workload"], "pairs": s["pairs"], "stage2_hits": s["stage2_hits"],
        "pairs_per_key_max": s["pairs_per_key"]["max"],
        "persistent": {k: round(v, 3) for k, v in s["schedules"]["persistent"].items() if k != "pairs_per_s"},
        "per_key": {k: round(v, 3) for k, v in s["schedules"]["per_key"].items() if k != "pairs_per_s"},
        "speedup_persistent_over_per_key": round(s["speedup_persistent_over_per_key"], 3),
        "timing": "CUDA events, 1 warm-up + 2 timed searches per schedule",
    }
    torch.cuda.empty_cache()
    log(f"batching stress done in {time.time() - t0:.1f}s")
    t0 = time.time()
    out["stage32"] = run_stage32(args)
    torch.cuda.empty_cache()
    log(f"stage 3.2 done in {time.time() - t0:.1f}s")
    t0 = time.time()
    saved = (args.query_proteins, args.bank2_proteins, args.scale)
    args.query_proteins, args.bank2_proteins = 250, 1_000_000
    try:
        q = run_query(args, steps=10, warmup=3, tiles=tiles)
    finally:
        args.query_proteins, args.bank2_proteins, args.scale = saved
    out["query_latency"] = {
        "workload": q["workload"], "pairs": q["pairs"], "records": q["records"],
        "plain_call_ms": round(q["search_ms"], 3), "planned_ms": round(q["plan_ms"], 3),
        "cuda_graph_ms": round(q["graph_ms"], 3), "stage_ms": q["stage_ms"],
        "resident_index_ms": round(q["resident_index_ms"], 1), "resident_windows_gb": q["resident_windows_gb"],
        "timing": "CUDA events, 3 warm-up + 10 timed searches per form",
    }
    torch.cuda.empty_cache()
    log(f"query latency done in {time.time() - t0:.1f}s")
    t0 = time.time()
    saved = args.requests
    args.requests = 60
    try:
        v = run_serving(args, rates=(20.0,), tiles=tiles)
    finally:
        args.requests = saved
    r = v["rows"][0]
    out["serving"] = {
        "workload": v["workload"], "rate_per_s": r["rate_per_s"],
        **{k: r[k] for k in r if k.startswith("p50") or k.startswith("p99") or k.startswith("pairs")},
        "batches": r["batches"], "mean_batch_requests": round(r["mean_batch_requests"], 2),
        "timing": "host wall clock from each request's arrival to its records, 60 requests",
    }
    log(f"serving done in {time.time() - t0:.1f}s")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="timed steps (the default spans about 1.5 s of the full-scale workload, enough for several clock samples)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (tests only)")
    ap.add_argument("--schedule", default="persistent", choices=["persistent", "per_key"])
    ap.add_argument("--cpu-steps", type=int, default=3,
                    help="cpu_baseline: timed oracle steps over the fixed key sample (about 4 s each on 16 cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary measurements (batching stress, resident-bank query latency)")
    ap.add_argument("--cpu-threads", type=int, default=None, help="oracle threads (default: every host core)")
    ap.add_argument("--tile-shape", default="auto", choices=["auto", "wide", "narrow", "narrow4", "narrow2", "narrow16"],
                    help="stage-2 tile shapes: by measured cost (default) or forced")
    ap.add_argument("--no-autotune", action="store_true", help="use the library's default tile costs")
    ap.add_argument("--wide-int16-cells", type=int, default=None, choices=[0, 12, 14, 16],
                    help="force the wide stage-2 kernel variant (default: the autotuner's pick)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "batching_stress", "tplastn", "plastx", "serving", "query", "stage32"],
                    help="the headline line is plastp_full; the others print their own lines")
    ap.add_argument("--s0", type=int, default=0,
                    help="Section 4.2 filter threshold for the headline workload (0: off, the bit-exact default; "
                         "53: the calibrated value)")
    ap.add_argument("--requests", type=int, default=60, help="serving: requests per arrival rate")
    ap.add_argument("--query-proteins", type=int, default=250, help="query: proteins of the query bank")
    ap.add_argument("--bank2-proteins", type=int, default=None,
                    help="bank-2 size of the headline workload (profiling captures use 10000)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        # the CPU oracle, on rank 0 only
        if rank != 0:
            return
        b1, _ = synth.workload(WORKLOAD, seed=1, scale=args.scale, n2=2)
        _, b2 = synth.workload(WORKLOAD, seed=shard_seed(0), scale=args.scale, n2=args.bank2_proteins)
        cb = run_oracle(b1, b2, args.steps, args.warmup, args.cpu_threads, s0=args.s0)
        line = {
            "impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["seconds_per_step"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": headline_config(b1, b2, cb["total_pairs"], args.scale, args.bank2_proteins, args.s0, world),
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return

    if args.workload != WORKLOAD:
        if rank == 0:
            fn = {"batching_stress": run_stress, "tplastn": run_tplastn, "plastx": run_plastx,
                  "serving": run_serving, "query": run_query, "stage32": run_stage32}[args.workload]
            print(json.dumps(fn(args)), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    result, banks = run_gpu(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_extras and args.scale == 1.0 and not args.bank2_proteins:
        from paper_0804_3643_gb300 import binding as B

        result["extras"] = run_extras(args, B.plast_get_tile_costs())
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            cb = run_oracle(banks[0], banks[1], args.cpu_steps, 0, args.cpu_threads, s0=args.s0)
            result["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
