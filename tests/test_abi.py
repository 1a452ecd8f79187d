"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/plast.h declares; host-only entry points behave."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def declared_functions():
    src = open(os.path.join(ROOT, "include", "plast.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(plast_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_0804_3643_gb300 import build

    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("plast_index_bank", "plast_translate6", "plast_ungapped", "plast_small_gapped", "plast_search"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(lib):
    from paper_0804_3643_gb300 import binding as B

    p = B.plast_default_params()
    assert p.as_dict() == dict(w=4, nl=22, nr=22, s1=38, lg=64, band=8, gap_open=11, gap_extend=1, s2=47, s0=0)
    assert B.plast_strerror(B.PLAST_E_CAPACITY) == "output capacity too small"
    assert B.plast_strerror(0) == "ok"
    B.plast_set_schedule(1)
    B.plast_set_schedule(0)
    with pytest.raises(B.PlastError):
        B.plast_set_schedule(7)
    B.plast_set_tile_shape(5)
    with pytest.raises(B.PlastError):
        B.plast_set_tile_shape(6)
    B.plast_set_tile_shape(0)
    c = B.plast_get_tile_costs()
    assert c["wide_slot"] > 0 and c["narrow_slot"] > 0
    with pytest.raises(B.PlastError):
        B.plast_set_tile_costs(dict(c, narrow_slot=-1.0))
    with pytest.raises(B.PlastError):
        B.plast_set_tile_costs(dict(c, wide_int16_cells=18))
    for n16 in (0, 12, 14, 16):
        B.plast_set_tile_costs(dict(c, wide_int16_cells=n16))
        assert B.plast_get_tile_costs()["wide_int16_cells"] == n16
    B.plast_set_tile_costs(dict(c, wide_tile=c["wide_tile"] + 1))
    assert B.plast_get_tile_costs()["wide_tile"] == c["wide_tile"] + 1
    B.plast_set_tile_costs(c)


def test_alloc_limit_setter(lib):
    from paper_0804_3643_gb300 import binding as B

    with pytest.raises(B.PlastError):
        B.plast_set_alloc_limit(-1)
    B.plast_set_alloc_limit(1 << 20)
    B.plast_set_alloc_limit(0)


def test_record_layouts_match_header():
    from paper_0804_3643_gb300 import binding as B

    assert B.HIT_DTYPE.itemsize == 20 and B.GAPPED_DTYPE.itemsize == 28
    assert ctypes.sizeof(B.plast_params) == 40
    assert ctypes.sizeof(B.plast_tile_costs) == 88
