"""plast_small_gapped_noalloc against the oracle and plast_small_gapped.

The no-allocation entry point serves callers that cannot let the library
allocate device memory (their GPU memory is already reserved by their own
allocator, or their request loop must not stall on or fail in an
allocation).  It runs the same stage-3.1 kernels on a fixed device scratch
array that keeps its contents between calls, so this test makes calls in a
row with different hit lists and requires each result to equal, byte for
byte, both the oracle's stage 3.1 of the same hits and what the allocating
entry point returns.  One call takes exactly the largest list the scratch
holds, and calls run with every library allocation made to fail, which
they must not notice.  The file is named to be collected last and builds
everything it needs, so it passes both alone in a fresh process and after
the other GPU tests.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_0804_3643_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_0804_3643_gb300 import binding as B
    from paper_0804_3643_gb300 import build

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    B.lib()
    b1, b2 = synth.workload("plastp_plain", seed=21, scale=0.2)
    d1 = B.DeviceBank.from_host(b1.codes, b1.seq_off)
    d2 = B.DeviceBank.from_host(b2.codes, b2.seq_off)
    g1 = B.plast_index_bank(d1.codes, d1.seq_off)
    g2 = B.plast_index_bank(d2.codes, d2.seq_off)
    # more hits than the default threshold gives, to fill much of the scratch
    hits = B.plast_ungapped(g1, g2, B.plast_default_params(s1=30))
    o1 = oracle.make_bank(b1.codes, b1.seq_off)
    o2 = oracle.make_bank(b2.codes, b2.seq_off)
    return B, g1, g2, hits, o1, o2


def noalloc(B, g1, g2, hits, params):
    out = torch.empty(max(hits.shape[0], 1) * B.GAPPED_BYTES, dtype=torch.uint8, device="cuda")
    got = B.plast_small_gapped_noalloc(g1, g2, hits, out, params)
    torch.cuda.synchronize()
    return got.cpu().numpy()


def want_of(B, g1, g2, o1, o2, hits, s2):
    """(oracle records, plast_small_gapped records) of ``hits`` as uint8 rows."""
    w = oracle.small_gapped(o1, o2, B.hits_numpy(hits), oracle.Params(s2=s2), threads=8)
    alloc = B.plast_small_gapped(g1, g2, hits, B.plast_default_params(s2=s2)).cpu().numpy()
    return w.view(np.uint8).reshape(-1, B.GAPPED_BYTES), alloc


def test_noalloc_matches_oracle_and_allocating_entry_point_on_two_calls(setup):
    B, g1, g2, hits, o1, o2 = setup
    n = hits.shape[0]
    assert 2000 < n <= B.NOALLOC_MAX_HITS
    # call 1: every hit, every record kept
    got = noalloc(B, g1, g2, hits, B.plast_default_params(s2=-10000))
    w, alloc = want_of(B, g1, g2, o1, o2, hits, -10000)
    assert w.shape[0] == n
    assert np.array_equal(got, w) and np.array_equal(got, alloc)
    # call 2: a different, shorter list at the default threshold; the scratch
    # still holds call 1's data
    sub = hits[n // 3: n // 3 + n // 2]
    got = noalloc(B, g1, g2, sub, B.plast_default_params())
    w, alloc = want_of(B, g1, g2, o1, o2, sub, 47)
    assert 0 < w.shape[0] < sub.shape[0]
    assert np.array_equal(got, w) and np.array_equal(got, alloc)


def test_noalloc_at_its_largest_list_with_allocations_failing(setup):
    B, g1, g2, hits, o1, o2 = setup
    # exactly PLAST_NOALLOC_MAX_HITS hits: the last slots of every scratch
    # array and the scan's scratch are used
    reps = -(-B.NOALLOC_MAX_HITS // hits.shape[0])
    big = hits.repeat(reps, 1)[: B.NOALLOC_MAX_HITS].contiguous()
    assert big.shape[0] == B.NOALLOC_MAX_HITS
    w, alloc = want_of(B, g1, g2, o1, o2, big, 40)
    assert 0 < w.shape[0] < big.shape[0]
    try:
        # every device allocation the library makes now fails; this entry
        # point makes none, so it still succeeds (twice in a row)
        B.plast_set_alloc_limit(1)
        for _ in range(2):
            got = noalloc(B, g1, g2, big, B.plast_default_params(s2=40))
            assert np.array_equal(got, w) and np.array_equal(got, alloc)
        with pytest.raises(B.PlastError) as e:
            B.plast_small_gapped(g1, g2, big, B.plast_default_params(s2=40))
        assert e.value.code == B.PLAST_E_OOM
    finally:
        B.plast_set_alloc_limit(0)


def test_noalloc_rejects_more_hits_than_its_scratch(setup):
    B, g1, g2, hits, o1, o2 = setup
    big = hits[:1].repeat(B.NOALLOC_MAX_HITS + 1, 1)
    out = torch.empty(B.GAPPED_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.PlastError) as e:
        B.plast_small_gapped_noalloc(g1, g2, big, out)
    assert e.value.code == B.PLAST_E_INVALID
    # the parameter checks are the allocating entry point's
    with pytest.raises(B.PlastError) as e:
        B.plast_small_gapped_noalloc(g1, g2, hits[:10], out, B.plast_default_params(s1=40000))
    assert e.value.code == B.PLAST_E_INVALID
