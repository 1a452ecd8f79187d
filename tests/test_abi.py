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


def prototypes():
    """{name: [parameter types]} of every function the header declares."""
    src = open(os.path.join(ROOT, "include", "plast.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(plast_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = [" ".join(p.split()) for p in m.group(2).split(",") if p.strip()]
        types = []
        for p in params:
            p = p.replace(" *", "*")
            toks = p.split(" ")
            # drop the parameter name (a trailing identifier after a type)
            if len(toks) > 1 and re.fullmatch(r"[A-Za-z_][A-Za-z0-9_]*", toks[-1]) and toks[-1] not in (
                    "int", "void", "int32_t", "int64_t"):
                toks = toks[:-1]
            types.append(" ".join(toks))
        out[m.group(1)] = [] if types == ["void"] else types
    return out


# The calls of the boundary with the parameter types the hot-path contract
# gives them (Section 3.2's problem statement: translate, index, ungapped,
# small gapped, search).
BOUNDARY = {
    "plast_translate6": ["const uint8_t*", "const int64_t*", "int32_t", "int8_t*", "int64_t", "int64_t*",
                         "int32_t*", "int64_t*", "void*"],
    "plast_index_bank": ["const int8_t*", "const int64_t*", "int32_t", "const plast_params*", "void*",
                         "plast_bank**"],
    "plast_bank_free": ["plast_bank*"],
    "plast_ungapped": ["const plast_bank*", "const plast_bank*", "const plast_params*", "plast_hit*", "int64_t",
                       "int64_t*", "void*"],
    "plast_small_gapped": ["const plast_bank*", "const plast_bank*", "const plast_params*", "const plast_hit*",
                           "int64_t", "plast_gapped*", "int64_t", "int64_t*", "void*"],
    "plast_search": ["const plast_bank*", "const plast_bank*", "const plast_params*", "plast_gapped*", "int64_t",
                     "int64_t*", "void*"],
    "plast_strerror": ["int"],
}


def test_boundary_signatures():
    protos = prototypes()
    for name, types in BOUNDARY.items():
        assert protos.get(name) == types, (name, protos.get(name))


def test_boundary_structs():
    src = open(os.path.join(ROOT, "include", "plast.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)

    def fields(name):
        m = re.search(r"typedef struct\s*\{([^}]*)\}\s*" + name + r"\s*;", src)
        assert m, name
        return " ".join(m.group(1).split())

    assert fields("plast_params") == "int32_t w, nl, nr, s1, lg, band, gap_open, gap_extend, s2;"
    assert fields("plast_hit") == "int32_t seq1, pos1, seq2, pos2; int16_t score; int8_t rlen, llen;"
    assert fields("plast_gapped") == ("int32_t seq1, pos1, seq2, pos2; int16_t score, ungapped; "
                                      "int16_t r_i, r_j, l_i, l_j;")


def test_binding_argument_counts_match_header(lib):
    from paper_0804_3643_gb300 import binding as B

    L = B.lib()
    for name, types in prototypes().items():
        f = getattr(L, name)
        if f.argtypes is not None:
            assert len(f.argtypes) == len(types), (name, len(f.argtypes), types)


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(lib):
    from paper_0804_3643_gb300 import binding as B

    p = B.plast_default_params()
    assert p.as_dict() == dict(w=4, nl=22, nr=22, s1=38, lg=64, band=8, gap_open=11, gap_extend=1, s2=47)
    assert B.plast_strerror(B.PLAST_E_CAPACITY) == "output capacity too small"
    assert B.plast_strerror(0) == "ok"
    assert B.plast_full_gapped_cells() >= 0
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
        for depth in (1, 2):
            B.plast_set_tile_costs(dict(c, wide_int16_cells=n16, wide_stage_depth=depth))
            got = B.plast_get_tile_costs()
            assert got["wide_int16_cells"] == n16 and got["wide_stage_depth"] == depth
    with pytest.raises(B.PlastError):
        B.plast_set_tile_costs(dict(c, wide_stage_depth=3))
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
    assert ctypes.sizeof(B.plast_params) == 36
    assert ctypes.sizeof(B.plast_tile_costs) == 88
