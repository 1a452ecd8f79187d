"""Stage-2 work list (host logic, no GPU): every bank-1 occurrence of every
key shared by both banks lies in exactly one tile; full wide tiles first,
the remainder wide or narrow by the cost model; costliest tiles first in the
persistent schedule, key order in the plain one."""
import math

import numpy as np
import pytest

from paper_0804_3643_gb300 import binding as B

NK = B.NKEYS
WIDE, NARROW = 0, 1
T1, NT1 = 128, 8


def offsets(counts):
    off = np.zeros(NK + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off


@pytest.fixture()
def costs():
    B.lib()
    saved = B.plast_get_tile_costs()
    c = dict(wide_slot=0.5, wide_tile=4000.0, narrow_slot=0.6, narrow_tile=1000.0, wide_int16_cells=14)
    B.plast_set_tile_costs(c)
    yield c
    B.plast_set_tile_costs(saved)
    B.plast_set_tile_shape(0)
    B.plast_set_schedule(0)


def random_counts(rng):
    n1 = rng.choice([0, 1, 3, 7, 8, 9, 15, 40, 100, 127, 128, 129, 255, 256, 300, 1000], size=NK)
    n2 = rng.choice([0, 1, 5, 50, 500, 5000, 50000], size=NK)
    return n1.astype(np.int64), n2.astype(np.int64)


def round_up(n, g):
    return -(-int(n) // g) * g


def tile_cost(c, shape, n2):
    # a CTA scores 128 (wide) or 1024 (narrow) bank-2 windows per pass
    if shape == WIDE:
        return c["wide_slot"] * T1 * round_up(n2, 128) + c["wide_tile"]
    return c["narrow_slot"] * NT1 * round_up(n2, 1024) + c["narrow_tile"]


def check_cover(tiles, k1, n1, n2):
    by_key = {}
    for key, first, rows, shape in tiles:
        assert shape in (WIDE, NARROW)
        assert 1 <= rows <= (T1 if shape == WIDE else NT1)
        by_key.setdefault(int(key), []).append((int(first), int(rows), int(shape)))
    for k in range(NK):
        if n1[k] == 0 or n2[k] == 0:
            assert k not in by_key
            continue
        t = sorted(by_key[k])
        assert t[0][0] == k1[k]
        for (f, r, _), (f2, _, _) in zip(t, t[1:]):
            assert f + r == f2
        assert t[-1][0] + t[-1][1] == k1[k + 1]
    return by_key


def test_cover_and_shapes_by_cost(costs):
    rng = np.random.default_rng(5)
    n1, n2 = random_counts(rng)
    k1, k2 = offsets(n1), offsets(n2)
    tiles = B.plast_stage2_tiles(k1, k2)
    by_key = check_cover(tiles, k1, n1, n2)
    for k, t in by_key.items():
        t = sorted(t)
        full = n1[k] // T1
        assert all(s == WIDE and r == T1 for _, r, s in t[:full])
        rest = t[full:]
        rem = n1[k] - full * T1
        if rem == 0:
            assert not rest
            continue
        want_narrow = math.ceil(rem / NT1) * tile_cost(costs, NARROW, n2[k]) < tile_cost(costs, WIDE, n2[k])
        if want_narrow:
            assert all(s == NARROW for _, _, s in rest) and len(rest) == math.ceil(rem / NT1)
        else:
            assert len(rest) == 1 and rest[0][2] == WIDE and rest[0][1] == rem
    # costliest first
    c = [tile_cost(costs, s, n2[key]) for key, _, _, s in tiles]
    assert all(a >= b for a, b in zip(c, c[1:]))
    # both shapes occur in this mix
    assert (tiles[:, 3] == WIDE).any() and (tiles[:, 3] == NARROW).any()


@pytest.mark.parametrize("shape", [1, 2])
def test_forced_shapes(costs, shape):
    rng = np.random.default_rng(6)
    n1, n2 = random_counts(rng)
    k1, k2 = offsets(n1), offsets(n2)
    B.plast_set_tile_shape(shape)
    tiles = B.plast_stage2_tiles(k1, k2)
    check_cover(tiles, k1, n1, n2)
    assert (tiles[:, 3] == (WIDE if shape == 1 else NARROW)).all()


def test_plain_schedule_keeps_key_order(costs):
    rng = np.random.default_rng(7)
    n1, n2 = random_counts(rng)
    B.plast_set_schedule(1)
    tiles = B.plast_stage2_tiles(offsets(n1), offsets(n2))
    keys = tiles[:, 0]
    assert (np.diff(keys) >= 0).all()
    firsts = tiles[:, 1]
    same = np.diff(keys) == 0
    assert (np.diff(firsts)[same] > 0).all()


def test_small_query_goes_narrow(costs):
    # a query bank with a few occurrences per key against a large bank
    n1 = np.full(NK, 3, dtype=np.int64)
    n2 = np.full(NK, 40000, dtype=np.int64)
    tiles = B.plast_stage2_tiles(offsets(n1), offsets(n2))
    assert (tiles[:, 3] == NARROW).all() and len(tiles) == NK


def test_bad_offsets(costs):
    k = offsets(np.ones(NK, dtype=np.int64))
    bad = k.copy()
    bad[10] = bad[11] + 1
    with pytest.raises(B.PlastError):
        B.plast_stage2_tiles(bad, k)
    with pytest.raises(ValueError):
        B.plast_stage2_tiles(k[:-1], k)
