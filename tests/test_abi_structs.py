"""The ctypes mirrors of the C-ABI structs in the Python binding have the sizes and
field offsets that the C compiler gives the declarations in include/ift.h (a small
host program compiled with gcc against the header; no GPU)."""

import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2305_15661_gb300 import ift

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = [("ift_config", ift.Config), ("ift_solve_info", ift.SolveInfo), ("ift_align_info", ift.AlignInfo)]


def _c_layouts(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ift.h"', "int main(void) {"]
    for cname, cls in STRUCTS:
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        name, field, val = ln.split()
        got[(name, field)] = int(val)
    return got


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ctypes_structs_match_the_header(tmp_path):
    got = _c_layouts(tmp_path)
    for cname, cls in STRUCTS:
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
