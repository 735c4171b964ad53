"""The C ABI library loads without a GPU and exports every symbol include/aderweno.h declares;
the Python binding declares a signature for each (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_1212_3585_gb300 as pg
from paper_1212_3585_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "aderweno.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(aw_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("aw_create", "aw_set_initial", "aw_step", "aw_advance_to", "aw_regrid", "aw_regrid_with_flags",
              "aw_read_cells", "aw_read_internal", "aw_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1212_3585_gb300 import build
        build.build()
    L = ctypes.CDLL(_lib.LIB_PATH)
    for n in declared():
        assert hasattr(L, n), n
    assert set(declared()) == set(_lib.SIGNATURES), set(declared()) ^ set(_lib.SIGNATURES)


def test_binding_loads_and_rejects_bad_config_without_gpu():
    L = _lib.load()
    assert L.aw_last_error() is not None
    cfg = pg.make_config(dim=4)
    h = ctypes.c_void_p()
    rc = L.aw_create(ctypes.byref(cfg), 0, ctypes.byref(h))
    assert rc == _lib.AW_EINVAL and b"dim" in L.aw_last_error()


def test_struct_layouts_match_header():
    # sizes implied by the header's field list (natural alignment)
    assert ctypes.sizeof(pg.AwConfig) == 4 * 6 + 8 * 2 + 8 * 6 + 4 * 6 + 4 * 2 + 8 * 4 + 4 * 4 + 8 * 3
    assert ctypes.sizeof(pg.AwCell) == 20
    assert ctypes.sizeof(pg.AwStats) == 8 * 10 + 8 * 2
