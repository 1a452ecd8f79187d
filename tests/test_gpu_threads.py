"""Calls from several host threads at once, each on its own stream: indexing,
stage 2 and whole searches give the oracle's results bit for bit (the
library's per-device state, stage timers and scratch are per call or per
thread; shared banks are read-only)."""
import threading

import numpy as np
import pytest
import torch

import oracle
from paper_0804_3643_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_0804_3643_gb300 import binding, build

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    binding.lib()
    yield binding


def same(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint8), b.view(np.uint8))


def run_threads(fs):
    out, errs = [None] * len(fs), []

    def body(i):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                out[i] = fs[i](s)
        except BaseException as e:  # reported on the main thread
            errs.append(e)

    ts = [threading.Thread(target=body, args=(i,)) for i in range(len(fs))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errs:
        raise errs[0]
    return out


def test_concurrent_index_and_search(B):
    b1, b2 = synth.workload("plastp_plain", seed=17, scale=0.5)
    q = synth.protein_bank(np.random.default_rng(18), 120)
    banks = [(b1.codes, b1.seq_off), (b2.codes, b2.seq_off), (q.codes, q.seq_off)]
    ob = [oracle.make_bank(c, o) for c, o in banks]
    jobs = [(0, 1), (1, 0), (2, 1), (0, 2)]
    want_h = [oracle.ungapped(ob[i], ob[j], threads=16) for i, j in jobs]
    want = [oracle.small_gapped(ob[i], ob[j], h) for (i, j), h in zip(jobs, want_h)]
    assert all(len(w) > 0 for w in want)

    def index(c, o):
        def f(s):
            d = B.DeviceBank.from_host(c, o)
            g = B.plast_index_bank(d.codes, d.seq_off, stream=s)
            s.synchronize()
            return g
        return f

    # three banks indexed at once
    g = run_threads([index(c, o) for c, o in banks])
    for gi, oi in zip(g, ob):
        key_off, pos = B.plast_bank_export_index(gi)
        assert np.array_equal(key_off.cpu().numpy(), oi.idx.key_off)
        assert np.array_equal(pos.cpu().numpy(), oi.idx.pos)

    def search(k):
        i, j = jobs[k]

        def f(s):
            res = []
            for _ in range(3):
                h = B.hits_numpy(B.plast_ungapped(g[i], g[j], stream=s))
                r, n = B.plast_search_ex(g[i], g[j], stream=s)
                res.append((h, B.gapped_numpy(r), n))
            return res
        return f

    # four searches at once, each three times
    for k, res in enumerate(run_threads([search(k) for k in range(len(jobs))])):
        for h, r, n in res:
            assert same(h, want_h[k])
            assert n == len(want_h[k]) and same(r, want[k])
