import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")
AA = "ARNDCQEGHILKMFPSTWYV"


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def golden(name: str) -> dict:
    """key: value lines of a fixture under tests/golden (comments dropped)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = v.strip()
    return out


def enc(s: str) -> np.ndarray:
    """Protein letters to codes 0..19 (A R N D C Q E G H I L K M F P S T W Y V), '*' = 20."""
    return np.array([20 if c == "*" else AA.index(c) for c in s], dtype=np.int8)


def bank_from(seqs):
    """(codes, seq_off) of a list of letter strings or code arrays."""
    arrs = [enc(s) if isinstance(s, str) else np.asarray(s, dtype=np.int8) for s in seqs]
    off = np.zeros(len(arrs) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(a) for a in arrs])
    codes = np.concatenate(arrs) if arrs else np.zeros(0, np.int8)
    return codes.astype(np.int8), off


@pytest.fixture(scope="session")
def rng():
    return np.random.default_rng(12345)
