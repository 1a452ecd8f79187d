"""Stage-2 work list (host logic, no GPU): every bank-1 occurrence of every
key shared by both banks lies in exactly one tile; full wide tiles first,
the remainder one wide tile or narrow tiles (16 rows while 16 remain, or 8
where those cost less per row, the last rows by the cheapest cover with 16,
8, 4 and 2) by the cost model; in the
persistent schedule wide tiles (one launch) before narrow tiles (another),
each costliest first; key order in the plain one."""
import math

import numpy as np
import pytest

from paper_0804_3643_gb300 import binding as B

NK = B.NKEYS
WIDE, NARROW, NARROW4, NARROW2, NARROW16 = 0, 1, 2, 3, 4
ROWS = {WIDE: 128, NARROW: 8, NARROW4: 4, NARROW2: 2, NARROW16: 16}
NAME = {WIDE: "wide", NARROW: "narrow", NARROW4: "narrow4", NARROW2: "narrow2", NARROW16: "narrow16"}
T1 = 128


def offsets(counts):
    off = np.zeros(NK + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off


@pytest.fixture()
def costs():
    B.lib()
    saved = B.plast_get_tile_costs()
    c = dict(wide_slot=0.5, wide_tile=4000.0, narrow_slot=0.6, narrow_tile=1000.0, narrow4_slot=0.8,
             narrow4_tile=900.0, narrow2_slot=1.1, narrow2_tile=800.0, narrow16_slot=0.5, narrow16_tile=1200.0,
             wide_int16_cells=12)
    B.plast_set_tile_costs(c)
    yield c
    B.plast_set_tile_costs(saved)
    B.plast_set_tile_shape(0)
    B.plast_set_schedule(0)


def random_counts(rng):
    n1 = rng.choice([0, 1, 3, 7, 8, 9, 15, 16, 17, 24, 40, 100, 127, 128, 129, 255, 256, 300, 1000], size=NK)
    n2 = rng.choice([0, 1, 5, 50, 500, 5000, 50000], size=NK)
    return n1.astype(np.int64), n2.astype(np.int64)


def round_up(n, g):
    return -(-int(n) // g) * g


def tile_cost(c, shape, n2):
    # a CTA scores 128 (wide) or 512 (narrow) bank-2 windows per pass
    name = NAME[shape]
    return c[name + "_slot"] * ROWS[shape] * round_up(n2, 128 if shape == WIDE else 512) + c[name + "_tile"]


def tail_cover(c, t, n2):
    """Cost of the cheapest cover of t < 16 rows by narrow tiles of 16, 8, 4
    and 2 rows, by brute force over multisets."""
    if t == 0:
        return 0.0
    best = None
    for a in range(0, 2):                  # tiles of 16
        for e in range(0, 3):              # tiles of 8
            for b in range(0, 5):          # tiles of 4
                for d in range(0, 9):      # tiles of 2
                    if 16 * a + 8 * e + 4 * b + 2 * d < t or a + e + b + d == 0:
                        continue
                    cost = (a * tile_cost(c, NARROW16, n2) + e * tile_cost(c, NARROW, n2)
                            + b * tile_cost(c, NARROW4, n2) + d * tile_cost(c, NARROW2, n2))
                    best = cost if best is None else min(best, cost)
    return best


def check_cover(tiles, k1, n1, n2):
    """Rows: every bank-1 occurrence of a shared key in exactly one row range;
    windows: for each row range, the bank-2 ranges of its pieces partition
    [0, n2) of the key's list in whole passes (the last piece ragged)."""
    by_key, pieces = {}, {}
    for key, first, rows, shape, vlo, vhi in tiles:
        assert shape in ROWS
        assert 1 <= rows <= ROWS[shape]
        assert 0 <= vlo < vhi <= n2[key]
        pieces.setdefault((int(key), int(first), int(rows), int(shape)), []).append((int(vlo), int(vhi)))
    for (key, first, rows, shape), v in pieces.items():
        v.sort()
        assert v[0][0] == 0 and v[-1][1] == n2[key]
        for (a, b), (a2, _) in zip(v, v[1:]):
            assert b == a2 and (b - a) % (128 if shape == WIDE else 512) == 0
        by_key.setdefault(key, []).append((first, rows, shape))
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
    # no SM count given: no list is cut
    assert (tiles[:, 4] == 0).all() and (tiles[:, 5] == n2[tiles[:, 0]]).all()
    for k, t in by_key.items():
        t = sorted(t)
        full = n1[k] // T1
        assert all(s == WIDE and r == T1 for _, r, s in t[:full])
        rest = t[full:]
        rem = n1[k] - full * T1
        if rem == 0:
            assert not rest
            continue
        # full tiles of 16 rows (of 8 where those cost less per row), then the
        # cheapest cover of the rest
        bulk = NARROW16 if tile_cost(costs, NARROW16, n2[k]) <= 2 * tile_cost(costs, NARROW, n2[k]) else NARROW
        br = ROWS[bulk]
        narrow_cost = (rem // br) * tile_cost(costs, bulk, n2[k]) + tail_cover(costs, rem % br, n2[k])
        if narrow_cost < tile_cost(costs, WIDE, n2[k]):
            shapes = [s_ for _, _, s_ in rest]
            assert shapes[: rem // br] == [bulk] * (rem // br)
            assert all(r == br for _, r, _ in rest[: rem // br])
            assert all(s_ != WIDE for s_ in shapes)
            assert abs(sum(tile_cost(costs, s_, n2[k]) for s_ in shapes) - narrow_cost) < 1e-6
        else:
            assert len(rest) == 1 and rest[0][2] == WIDE and rest[0][1] == rem
    # wide tiles first (one launch), then narrow ones (another), each costliest first
    wide = tiles[:, 3] == WIDE
    n_wide = int(wide.sum())
    assert wide[:n_wide].all() and not wide[n_wide:].any()
    for part in (tiles[:n_wide], tiles[n_wide:]):
        c = [tile_cost(costs, s, hi - lo) for _, _, _, s, lo, hi in part]
        assert all(a >= b for a, b in zip(c, c[1:]))
    # every shape occurs in this mix
    for shape in ROWS:
        assert (tiles[:, 3] == shape).any(), shape


@pytest.mark.parametrize("shape", [1, 2, 3, 4, 5])
def test_forced_shapes(costs, shape):
    rng = np.random.default_rng(6)
    n1, n2 = random_counts(rng)
    k1, k2 = offsets(n1), offsets(n2)
    B.plast_set_tile_shape(shape)
    tiles = B.plast_stage2_tiles(k1, k2)
    check_cover(tiles, k1, n1, n2)
    assert (tiles[:, 3] == shape - 1).all()


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
    n2 = np.full(NK, 40000, dtype=np.int64)
    for n, shape in [(1, NARROW2), (2, NARROW2), (4, NARROW4), (8, NARROW), (16, NARROW16)]:
        tiles = B.plast_stage2_tiles(offsets(np.full(NK, n, dtype=np.int64)), offsets(n2))
        assert (tiles[:, 3] == shape).all() and len(tiles) == NK, n


def test_few_tiles_cut_long_lists(costs):
    # a two-protein query: a few hundred keys with one occurrence each against
    # long bank-2 lists, fewer tiles than the narrow launch's CTAs
    rng = np.random.default_rng(8)
    n1 = np.zeros(NK, dtype=np.int64)
    n1[rng.choice(NK, 300, replace=False)] = 1
    n2 = rng.integers(1000, 60000, size=NK).astype(np.int64)
    k1, k2 = offsets(n1), offsets(n2)
    whole = B.plast_stage2_tiles(k1, k2)
    cut = B.plast_stage2_tiles(k1, k2, n_sms=152)
    assert len(whole) == 300 and len(cut) > 2 * 152
    check_cover(cut, k1, n1, n2)
    cost = [tile_cost(costs, s, hi - lo) for _, _, _, s, lo, hi in cut]
    assert all(a >= b for a, b in zip(cost, cost[1:]))
    # no piece above twice the target of a quarter of a CTA's share
    assert max(cost) <= 2 * sum(cost) / (4 * 2 * 152) + tile_cost(costs, NARROW2, 512)
    # a large mix has tiles enough: nothing is cut
    n1, n2 = random_counts(rng)
    k1, k2 = offsets(n1), offsets(n2)
    assert (B.plast_stage2_tiles(k1, k2, n_sms=152) == B.plast_stage2_tiles(k1, k2)).all()


def test_bad_offsets(costs):
    k = offsets(np.ones(NK, dtype=np.int64))
    bad = k.copy()
    bad[10] = bad[11] + 1
    with pytest.raises(B.PlastError):
        B.plast_stage2_tiles(bad, k)
    with pytest.raises(ValueError):
        B.plast_stage2_tiles(k[:-1], k)
