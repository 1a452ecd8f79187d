"""Planned search (preallocated, no host synchronisation) and its CUDA-graph
replay give the oracle's records, the same as plast_search; exceeding either
limit reports PLAST_E_CAPACITY."""
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
    binding.plast_set_schedule(0)
    return binding


@pytest.fixture(scope="module")
def banks(B):
    b1, b2 = synth.workload("plastp_plain", seed=3, scale=0.5)
    out = []
    for b in (b1, b2):
        d = B.DeviceBank.from_host(b.codes, b.seq_off)
        out.append(B.plast_index_bank(d.codes, d.seq_off))
    o1 = oracle.make_bank(b1.codes, b1.seq_off)
    o2 = oracle.make_bank(b2.codes, b2.seq_off)
    hits = oracle.ungapped(o1, o2, threads=16)
    want = oracle.small_gapped(o1, o2, hits)
    return out[0], out[1], len(hits), want


def test_plan_run_and_graph_replay(B, banks):
    g1, g2, n_hits, want = banks
    assert len(want) > 50
    plan = B.Plan(g1, g2, max_hits=2 * n_hits + 1000, max_records=len(want) + 100)
    plan.run()
    recs, nu = plan.result()
    assert nu == n_hits
    got = B.gapped_numpy(recs)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8))
    ref, nu2 = B.plast_search_ex(g1, g2)
    assert nu2 == n_hits and torch.equal(ref, recs)

    st = torch.cuda.Stream()
    plan.capture(st)
    for _ in range(2):
        plan.records.fill_(0xAB)
        plan.launch(st)
        recs, nu = plan.result(st)
        assert nu == n_hits
        assert np.array_equal(B.gapped_numpy(recs).view(np.uint8), want.view(np.uint8))
    plan.free()


def test_plan_capacity_errors(B, banks):
    g1, g2, n_hits, want = banks
    small_hits = B.Plan(g1, g2, max_hits=n_hits // 2, max_records=len(want) + 100)
    small_hits.run()
    with pytest.raises(B.PlastError) as e:
        small_hits.result()
    assert e.value.code == B.PLAST_E_CAPACITY and e.value.needed == n_hits
    small_recs = B.Plan(g1, g2, max_hits=n_hits + 10, max_records=len(want) - 1)
    small_recs.run()
    with pytest.raises(B.PlastError) as e:
        small_recs.result()
    assert e.value.code == B.PLAST_E_CAPACITY and e.value.needed == len(want)
    # the records that fit are distinct records of the full result, in order
    got = B.gapped_numpy(small_recs.records[: (len(want) - 1) * B.GAPPED_BYTES].view(-1, B.GAPPED_BYTES))
    full = {r.tobytes() for r in want}
    assert all(r.tobytes() in full for r in got) and len({r.tobytes() for r in got}) == len(got)
    key = [(int(r["seq1"]), int(r["pos1"]), int(r["seq2"]), int(r["pos2"])) for r in got]
    assert key == sorted(key)
    with pytest.raises(B.PlastError):
        B.Plan(g1, g2, max_hits=0, max_records=11)


def test_plan_with_filter(B, banks):
    # Section 4.2's filter inside a planned search and its graph replay
    g1, g2, n_hits, _ = banks
    b1, b2 = synth.workload("plastp_plain", seed=3, scale=0.5)
    o1 = oracle.make_bank(b1.codes, b1.seq_off)
    o2 = oracle.make_bank(b2.codes, b2.seq_off)
    prm_o = oracle.Params(s0=B.PLAST_FILTER_S0)
    hits = oracle.ungapped(o1, o2, prm_o, threads=16)
    want = oracle.small_gapped(o1, o2, hits)
    assert 0 < len(hits) < n_hits
    plan = B.Plan(g1, g2, max_hits=n_hits + 100, max_records=len(want) + 100, s0=B.PLAST_FILTER_S0)
    plan.run()
    recs, nu = plan.result()
    assert nu == len(hits)
    assert np.array_equal(B.gapped_numpy(recs).view(np.uint8), want.view(np.uint8))
    s = torch.cuda.Stream()
    plan.capture(s)
    for _ in range(2):
        plan.launch(s)
        s.synchronize()
        recs, nu = plan.result(s)
        assert nu == len(hits)
        assert np.array_equal(B.gapped_numpy(recs).view(np.uint8), want.view(np.uint8))
