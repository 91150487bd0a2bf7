"""The ctypes structures of the Python binding must match the C structures of
include/dbbc.h field by field: every struct's size and every field's offset,
as a C compiler on this machine lays them out (no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2609_21848_gb300 as dbbc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {"dbbc_graph_info": dbbc.GraphInfo, "dbbc_count_profile": dbbc.CountProfile, "dbbc_tuning": dbbc.Tuning}


def c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dbbc.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        struct, key, val = line.split()
        got[(struct, key)] = int(val)
    return got


def test_binding_structs_match_the_header(tmp_path):
    c = c_layout(tmp_path)
    for cname, py in STRUCTS.items():
        assert ctypes.sizeof(py) == c[(cname, "size")], cname
        for fname, _ in py._fields_:
            assert getattr(py, fname).offset == c[(cname, fname)], (cname, fname)
