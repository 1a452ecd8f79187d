"""plast_small_gapped_noalloc against plast_small_gapped.

The no-allocation entry point serves callers that cannot let the library
allocate device memory (their GPU memory is already reserved by their own
allocator, or their request loop must not stall on or fail in an
allocation).  It runs the same stage-3.1 kernels on a fixed device scratch
array that keeps its contents between calls, so this test makes two calls
in a row with different hit lists and requires each result to equal, byte
for byte, what the allocating entry point returns for the same hits.  The
file is named to be collected last and builds everything it needs, so it
passes both alone in a fresh process and after the other GPU tests.
"""
import numpy as np
import pytest
import torch

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
    return B, g1, g2, hits


def run_both(B, g1, g2, hits, params):
    want = B.plast_small_gapped(g1, g2, hits, params)
    out = torch.empty(max(hits.shape[0], 1) * B.GAPPED_BYTES, dtype=torch.uint8, device="cuda")
    got = B.plast_small_gapped_noalloc(g1, g2, hits, out, params)
    torch.cuda.synchronize()
    return got.cpu().numpy(), want.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_on_two_calls(setup):
    B, g1, g2, hits = setup
    n = hits.shape[0]
    assert 2000 < n <= B.NOALLOC_MAX_HITS
    every = B.plast_default_params(s2=-10000)
    # call 1: every hit, every record kept
    got, want = run_both(B, g1, g2, hits, every)
    assert want.shape[0] == n
    assert np.array_equal(got, want)
    # call 2: a different, shorter list at the default threshold; the scratch
    # still holds call 1's data
    sub = hits[n // 3: n // 3 + n // 2]
    got, want = run_both(B, g1, g2, sub, B.plast_default_params())
    assert 0 < want.shape[0] < sub.shape[0]
    assert np.array_equal(got, want)


def test_noalloc_rejects_more_hits_than_its_scratch(setup):
    B, g1, g2, hits = setup
    big = hits[:1].repeat(B.NOALLOC_MAX_HITS + 1, 1)
    out = torch.empty(B.GAPPED_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.PlastError) as e:
        B.plast_small_gapped_noalloc(g1, g2, big, out)
    assert e.value.code == B.PLAST_E_INVALID
