"""The C ABI library loads without a GPU and exports every symbol include/aderweno.h declares;
the Python binding declares a signature for each, whose argument and return types match the
header's prototypes in width and pointee; the ctypes structures have the header's layouts (no
compute calls here)."""
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


def test_struct_layouts_match_header(tmp_path):
    """sizes and field offsets of the ctypes structures equal those the C compiler gives the
    header's structures"""
    structs = {"aw_config": pg.AwConfig, "aw_stats": pg.AwStats, "aw_cell": pg.AwCell,
               "aw_srv_info": pg.AwSrvInfo, "aw_srv_summary": pg.AwSrvSummary,
               "aw_launch_params": _lib.AwLaunchParams, "aw_tune_entry": _lib.AwTuneEntry}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "aderweno.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {tuple(l.split()[:2]): int(l.split()[2]) for l in got if l}
    for cname, py in structs.items():
        assert c_layout[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert c_layout[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_launch_params_roundtrip_without_gpu():
    """the launch-shape rules are host state: read, changed, rejected when out of range, restored"""
    before = pg.get_launch_params()
    assert before == {"pass_min_cells": 4096, "tile8_min_cells": 20000, "small_ctas_per_sm": 2,
                      "fuse_flux_update": 1, "autotune": 1, "persistent": 0, "graph_steps": 0}
    pg.set_launch_params(small_ctas_per_sm=0, pass_min_cells=0, fuse_flux_update=0, autotune=0, persistent=1,
                         graph_steps=1)
    assert pg.get_launch_params() == {"pass_min_cells": 0, "tile8_min_cells": 20000, "small_ctas_per_sm": 0,
                                      "fuse_flux_update": 0, "autotune": 0, "persistent": 1, "graph_steps": 1}
    with pytest.raises(pg.AwError):
        pg.set_launch_params(small_ctas_per_sm=65)
    with pytest.raises(pg.AwError):
        pg.set_launch_params(fuse_flux_update=2)
    with pytest.raises(pg.AwError):
        pg.set_launch_params(autotune=-1)
    with pytest.raises(pg.AwError):
        pg.set_launch_params(persistent=3)
    with pytest.raises(pg.AwError):
        pg.set_launch_params(graph_steps=2)
    pg.set_launch_params(**before)
    assert pg.get_launch_params() == before


def prototypes():
    """(return type, name, [parameter types]) of every function the header declares"""
    src = open(os.path.join(ROOT, "include", "aderweno.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"#[^\n]*", "", src)
    out = []
    for m in re.finditer(r"([A-Za-z_][\w \*]*?)\b(aw_\w+)\s*\(([^;{]*)\)\s*;", src):
        ret, name, params = m.group(1).strip(), m.group(2), m.group(3)
        types = []
        for p in [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]:
            t = re.sub(r"\b\w+$", "", p).strip()          # drop the parameter name
            types.append(re.sub(r"\s+", " ", t.replace("*", " * ")).strip())
        out.append((re.sub(r"\s+", " ", ret.replace("*", " * ")).strip(), name, types))
    return out


SCALARS = {"int": ctypes.c_int, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double,
           "uintptr_t": ctypes.c_size_t}
STRUCTS = {"aw_config": pg.AwConfig, "aw_stats": pg.AwStats, "aw_cell": pg.AwCell, "aw_srv_info": pg.AwSrvInfo,
           "aw_srv_summary": pg.AwSrvSummary, "aw_launch_params": _lib.AwLaunchParams,
           "aw_tune_entry": _lib.AwTuneEntry, "int8_t": ctypes.c_int8, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double}
OPAQUE = {"aw_solver", "aw_server"}


def compatible(ctype, ct):
    """does the ctypes type ct pass the C type ctype (spelled with spaces around '*')?"""
    words = [w for w in ctype.split() if w != "const"]
    stars = words.count("*")
    base = words[0]
    if stars == 0:
        return SCALARS.get(base) is ct and ct is not None
    if ct is ctypes.c_void_p:                       # any pointer may travel as void*
        return base in OPAQUE and stars == 1 or base not in OPAQUE
    if stars == 1 and base == "char":
        return ct is ctypes.c_char_p
    if not hasattr(ct, "_type_"):
        return False
    inner = ct._type_
    if stars == 2 and base in OPAQUE:               # aw_solver** / aw_solver* const*
        return inner is ctypes.c_void_p
    return stars == 1 and STRUCTS.get(base) is inner


def test_binding_signatures_match_the_header():
    protos = prototypes()
    assert {p[1] for p in protos} == set(declared())
    for ret, name, params in protos:
        restype, argtypes = _lib.SIGNATURES[name]
        assert len(argtypes) == len(params), (name, params)
        for ctype, ct in zip(params, argtypes):
            assert compatible(ctype, ct), (name, ctype, ct)
        if ret == "void":
            assert restype is None, name
        elif ret == "const char *":
            assert restype is ctypes.c_char_p, name
        else:
            assert restype is SCALARS[ret], (name, ret, restype)


def test_tuning_state_without_gpu():
    """the autotuner's table is host state: empty after a reset; a null count is rejected"""
    pg.reset_tuning()
    assert pg.get_tuning() == []
    L = _lib.load()
    assert L.aw_get_tuning(None, 0, None) == _lib.AW_EINVAL
    n = ctypes.c_int32(-5)
    assert L.aw_get_tuning(None, -1, ctypes.byref(n)) == _lib.AW_EINVAL
    assert L.aw_get_tuning(None, 0, ctypes.byref(n)) == _lib.AW_OK and n.value == 0
