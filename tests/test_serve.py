"""Serving loop: admission, batching and memory accounting on the CPU with a
stand-in executor; on the GPU, each request's records are the same alone and
in a batch with others (continuous batching changes scheduling, not
results)."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_0804_3643_gb300 import serve, synth


def make_requests(n, seed, max_prot=20, rate=200.0):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    out = []
    for i in range(n):
        b = synth.random_protein_bank(rng, int(rng.integers(1, max_prot + 1)))
        out.append(serve.Request(i, float(t[i]), b.codes, b.seq_off))
    return out


class FakeExecutor:
    """Result of a request = sum of its codes per sequence; sleeps in
    proportion to the batch so batches overlap in time."""

    def __init__(self):
        self.lock = threading.Lock()
        self.batch_sizes = []

    def execute(self, reqs):
        with self.lock:
            self.batch_sizes.append(sum(r.n_seqs for r in reqs))
        codes, off, first = serve.merge_queries(reqs)
        time.sleep(0.002 + 0.0001 * len(codes) / 100)
        per_seq = np.add.reduceat(codes.astype(np.int64), off[:-1]) if len(codes) else np.zeros(0)
        res = [per_seq[first[q]:first[q + 1]] for q in range(len(reqs))]
        return res, int(len(codes))

    @staticmethod
    def mem_of(reqs):
        return 1000 * sum(r.n_seqs for r in reqs)


def test_merge_and_split_round_trip():
    reqs = make_requests(5, 1)
    codes, off, first = serve.merge_queries(reqs)
    assert first[-1] == sum(r.n_seqs for r in reqs) == len(off) - 1
    dt = np.dtype([("seq1", "<i4"), ("x", "<i4")])
    recs = np.zeros(len(off) - 1, dtype=dt)
    recs["seq1"] = np.arange(len(off) - 1)
    recs["x"] = np.arange(len(off) - 1) * 10
    parts = serve.split_records(recs, first)
    for q, r in enumerate(reqs):
        assert (parts[q]["seq1"] == np.arange(r.n_seqs)).all()
        assert (parts[q]["x"] == (first[q] + np.arange(r.n_seqs)) * 10).all()


@pytest.mark.parametrize("slots,budget", [(1, 10 ** 9), (3, 10 ** 9), (4, 25_000)])
def test_admission_batching_and_budget(slots, budget):
    ex = FakeExecutor()
    srv = serve.Server(ex.execute, ex.mem_of, slots=slots, mem_budget=budget, max_batch_seqs=30,
                       max_batch_requests=8)
    reqs = make_requests(60, 2)
    srv.run(reqs, realtime=True, timeout=60)
    # every request served exactly once, with its own result
    for r in reqs:
        assert r.done >= r.admitted >= r.arrival - 1e-6
        per_seq = np.add.reduceat(r.codes.astype(np.int64), r.seq_off[:-1])
        assert np.array_equal(r.result, per_seq)
    assert sum(len(b.requests) for b in srv.batches) == len(reqs)
    assert srv.peak_busy <= slots
    # a batch stays within the limits unless one request alone exceeds them
    for b in srv.batches:
        assert len(b.requests) <= 8
        seqs = sum(r.n_seqs for r in b.requests)
        assert seqs <= 30 or len(b.requests) == 1
    # the budget holds whenever more than one batch is in flight
    assert srv.peak_mem <= max(budget, max(b.mem_bytes for b in srv.batches))
    s = serve.latency_summary(reqs, sum(b.pairs for b in srv.batches), 1.0)
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_requests_arriving_while_busy_are_batched_together():
    ex = FakeExecutor()
    srv = serve.Server(ex.execute, ex.mem_of, slots=1, max_batch_seqs=10_000, max_batch_requests=100)
    reqs = make_requests(40, 3, rate=5000.0)  # arrivals much faster than service
    srv.run(reqs, realtime=True, timeout=60)
    assert len(srv.batches) < len(reqs)
    assert max(len(b.requests) for b in srv.batches) > 1


@pytest.mark.gpu
def test_gpu_result_same_alone_and_in_the_mix():
    import torch

    from paper_0804_3643_gb300 import build

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    rng = np.random.default_rng(8)
    bank = synth.protein_bank(rng, 3000)
    ex = serve.GpuExecutor(bank.codes, bank.seq_off)
    # requests: random proteins plus mutated copies of resident proteins
    reqs = []
    for i in range(12):
        b = synth.random_protein_bank(rng, int(rng.integers(1, 30)))
        seqs = [b.seq(k) for k in range(b.n_seqs)]
        seqs += [synth.mutate(rng, bank.seq(int(rng.integers(0, bank.n_seqs))), 0.7) for _ in range(3)]
        lens = np.array([len(x) for x in seqs])
        off = np.zeros(len(seqs) + 1, dtype=np.int64)
        off[1:] = np.cumsum(lens)
        reqs.append(serve.Request(i, 0.002 * i, np.concatenate(seqs).astype(np.int8), off))
    srv = serve.Server(ex.execute, ex.mem_of, slots=2, max_batch_seqs=60, max_batch_requests=5)
    srv.run(reqs, realtime=False, timeout=300)
    assert max(len(b.requests) for b in srv.batches) > 1
    n_rec = 0
    for r in reqs:
        alone = ex.alone(r)
        assert np.array_equal(r.result.view(np.uint8), alone.view(np.uint8))
        n_rec += len(alone)
    assert n_rec > 0
    # the same requests served with their stage-3.2 alignments: alone = in
    # the mix, and equal to the oracle's stage 3.2 of the request's records
    ex.full_gapped = True
    for r in reqs:
        r.result = None
    srv = serve.Server(ex.execute, ex.mem_of, slots=2, max_batch_seqs=60, max_batch_requests=5)
    srv.run(reqs, realtime=False, timeout=300)
    assert max(len(b.requests) for b in srv.batches) > 1
    o2 = oracle.make_bank(bank.codes, bank.seq_off)
    n_al = 0
    for r in reqs:
        alone = ex.alone(r)
        assert np.array_equal(r.result.view(np.uint8), alone.view(np.uint8))
        o1 = oracle.make_bank(r.codes, r.seq_off)
        want = oracle.full_gapped(o1, o2, oracle.small_gapped(o1, o2, oracle.ungapped(o1, o2)))
        assert np.array_equal(alone.view(np.uint8), want.view(np.uint8))
        n_al += len(alone)
    assert n_al > 0
