"""The C-ABI library loads and exports every function include/*.h declares.

No compute call is made here: this runs without a GPU.
"""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from conftest import ROOT


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(pp_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for want in ("pp_iblt_create", "pp_iblt_insert", "pp_iblt_decode", "pp_peel_kcore",
                 "pp_status_string", "pp_last_error"):
        assert want in names


def test_library_exports_every_declared_function(ppeel_lib):
    from paper_1302_7014_b300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        getattr(ppeel_lib, n)


def test_binding_declares_what_the_header_declares(ppeel_lib):
    import importlib
    import importlib.util
    for mod in ("paper_1302_7014_b300.batch", "paper_1302_7014_b300.server", "paper_1302_7014_b300.tune"):
        if importlib.util.find_spec(mod) is not None:
            importlib.import_module(mod)   # declares its entry points
    from paper_1302_7014_b300 import _lib
    assert set(declared_functions()) <= set(_lib.exported_symbols())


def test_host_only_calls(ppeel_lib):
    import paper_1302_7014_b300 as pp
    assert ppeel_lib.pp_status_string(3) == b"PP_ERR_CAPACITY"
    o = pp.options()
    assert o.block == 256 and o.max_rounds == 65535 and o.host_loop == 0
    assert ppeel_lib.pp_last_error() is not None


def test_struct_layouts_match_header(ppeel_lib, tmp_path):
    # offsets as the C compiler lays them out from include/ppeel.h vs the ctypes mirror
    from paper_1302_7014_b300 import _lib
    structs = {"pp_cell": _lib.Cell, "pp_options": _lib.Options,
               "pp_decode_result": _lib.DecodeResult, "pp_peel_result": _lib.PeelResult}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ppeel.h"', "int main(void){"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        a, b, c = line.split()
        got[(a, b)] = int(c)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_product_path_does_not_touch_the_oracle():
    # the package must never import, load or run anything under oracle/
    pkg = os.path.join(ROOT, "paper_1302_7014_b300")
    for p in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isfile(p) and p.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            src = open(p).read()
            assert "import oracle" not in src and "from oracle" not in src, p
            assert "liboracle" not in src and "peel_oracle" not in src, p


def test_workspace_size_host_only(ppeel_lib):
    import paper_1302_7014_b300 as pp
    small = pp.workspace_size(1 << 20, 3, 1000)
    assert small["table"] == 32 << 20   # 32-byte cells
    # below 2^21 cells nothing is binned: only what create allocates
    assert small["peak"] == small["table"] + small["fixed"]
    big = pp.workspace_size(1 << 24, 3, int(0.75 * (1 << 24)))
    assert big["table"] == 32 << 24 and big["fixed"] > 16 << 24
    assert big["peak"] > big["table"] + big["fixed"] + 12 * 3 * int(0.75 * (1 << 24))
    # binned=2 switches the binning off
    plain = pp.workspace_size(1 << 24, 3, int(0.75 * (1 << 24)), pp.options(binned=2))
    assert plain["peak"] == plain["table"] + plain["fixed"]
    with pytest.raises(pp.PPError):
        pp.workspace_size(10, 9)


def test_cell_dtype_matches_the_header(ppeel_lib):
    # the numpy view of a copied table has pp_cell's size and field offsets
    import numpy as np
    import paper_1302_7014_b300 as pp
    from paper_1302_7014_b300 import _lib
    dt = np.dtype(pp.CELL_DTYPE)
    assert dt.itemsize == ctypes.sizeof(_lib.Cell) == 32
    for name, _ in _lib.Cell._fields_:
        assert dt.fields[name][1] == getattr(_lib.Cell, name).offset, name
    raw = np.zeros(3, dt)
    raw["count"] = [-1, 0, 7]
    raw["chk_xor"] = [1, 2, 3]
    out = pp.unpack_cells(raw.tobytes())
    assert out["count"].tolist() == [-1, 0, 7] and out["chk_xor"].tolist() == [1, 2, 3]
