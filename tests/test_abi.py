"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/hb.h declares (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(hb_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["hb_init", "hb_query", "hb_build_blocks", "hb_diag", "hb_classify", "hb_destroy", "hb_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1709_03005_gb300 import build_ext, hb
    path = build_ext.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(hb.EXPORTS) <= set(_declared())


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1709_03005_gb300 import hb
    import pytest
    saved = hb._lib
    hb._lib = None
    try:
        with pytest.raises(RuntimeError):
            hb.load(str(tmp_path / "missing.so"))
    finally:
        hb._lib = saved


def test_struct_layouts_match_the_binding(tmp_path):
    """Every structure the binding mirrors (ctypes structures and the numpy
    record of hb_pair) has the header's size and field offsets (a C program
    built with the host compiler prints them)."""
    import shutil
    import subprocess
    import pytest
    from paper_1709_03005_gb300 import hb
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = [hb.hb_group, hb.hb_problem, hb.hb_options, hb.hb_layout, hb.hb_blocks, hb.hb_stats,
               hb.hb_mlp_weights, hb.hb_mlp_dataset]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hb.h"', "int main(void) {"]
    for S in structs:
        name = S.__name__
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in S._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    pair = hb.PAIR_DTYPE
    lines.append('    printf("hb_pair size %zu\\n", sizeof(hb_pair));')
    for field in pair.names:
        lines.append(f'    printf("hb_pair {field} %zu\\n", offsetof(hb_pair, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, key, value = line.split()
        got[(name, key)] = int(value)
    for S in structs:
        name = S.__name__
        assert got[(name, "size")] == ctypes.sizeof(S), name
        for field, _ in S._fields_:
            assert got[(name, field)] == getattr(S, field).offset, (name, field)
    # the classification records, read as a numpy structured array
    assert got[("hb_pair", "size")] == pair.itemsize
    for field in pair.names:
        assert got[("hb_pair", field)] == pair.fields[field][1], field
