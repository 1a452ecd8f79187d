"""Randomised parity: many small seeded workloads, each with its own
composition (planted homologs, low-complexity runs, very short and very long
proteins) and its own parameters drawn inside their valid ranges, through
the whole path on the GPU (stage 0, stages 1-2, stage 3.1 and stage 3.2)
against the oracle, byte for byte.  A case that fails names its seed."""
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
    return binding


def case(seed: int):
    """(bank 1, bank 2, parameters, drop-off) of one random case."""
    rng = np.random.default_rng(1000 + seed)
    n1, n2 = int(rng.integers(2, 60)), int(rng.integers(2, 400))
    b1 = synth.protein_bank(rng, n1, lowcomplex_frac=float(rng.choice([0.0, 0.0, 0.3])))
    b2 = synth.protein_bank(rng, n2, homolog_source=b1, planted_frac=float(rng.uniform(0.0, 0.5)),
                            lowcomplex_frac=float(rng.choice([0.0, 0.0, 0.2])))
    if seed % 5 == 0:  # a few very short sequences (shorter than a seed word)
        extra = [np.array(rng.integers(0, 20, int(rng.integers(1, 5))), dtype=np.int8) for _ in range(3)]
        seqs = [b2.seq(i) for i in range(b2.n_seqs)] + extra
        off = np.zeros(len(seqs) + 1, dtype=np.int64)
        np.cumsum([len(q) for q in seqs], out=off[1:])
        b2 = synth.SynthBank(np.concatenate(seqs).astype(np.int8), off)
    # (gap costs of BLAST's usual range: with nearly free gaps the alignments
    # of the planted homologs break into more gap-free segments per pair of
    # sequences than stage 3.2 keeps, PLAST_E_CAPACITY; the edge costs have
    # their own tests)
    p = dict(s1=int(rng.integers(20, 50)), s2=int(rng.integers(25, 70)), gap_open=int(rng.integers(5, 16)),
             gap_extend=int(rng.integers(1, 4)))
    return b1, b2, p, int(rng.integers(0, 80))


@pytest.mark.parametrize("seed", range(24))
def test_random_case(B, seed):
    b1, b2, p, x = case(seed)
    d1 = B.DeviceBank.from_host(b1.codes, b1.seq_off)
    d2 = B.DeviceBank.from_host(b2.codes, b2.seq_off)
    g1, g2 = B.plast_index_bank(d1.codes, d1.seq_off), B.plast_index_bank(d2.codes, d2.seq_off)
    o1, o2 = oracle.make_bank(b1.codes, b1.seq_off), oracle.make_bank(b2.codes, b2.seq_off)
    prm = oracle.Params(**p)
    gp = B.plast_default_params(**p)
    want_h = oracle.ungapped(o1, o2, prm)
    assert np.array_equal(B.hits_numpy(B.plast_ungapped(g1, g2, gp)).view(np.uint8), want_h.view(np.uint8)), seed
    want_g = oracle.small_gapped(o1, o2, want_h, prm)
    recs = B.plast_search(g1, g2, gp)
    assert np.array_equal(B.gapped_numpy(recs).view(np.uint8), want_g.view(np.uint8)), seed
    want_a, want_ext = oracle.full_gapped(o1, o2, want_g, prm, x=x, s3=p["s2"], return_extended=True)
    al, ext = B.plast_full_gapped(g1, g2, recs, gp, xdrop=x, s3=p["s2"])
    assert ext == want_ext, seed
    assert np.array_equal(B.alignments_numpy(al).view(np.uint8), want_a.view(np.uint8)), seed
