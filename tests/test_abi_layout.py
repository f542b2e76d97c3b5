"""The binding's ctypes mirrors of fsp_config, fsp_block, fsp_link and fsp3_block have the C layout of
include/fsp.h: gcc prints sizeof and offsetof of every field from the header, and the
binding's structures must agree (CPU; a mismatch would hand the library shifted arguments)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1810_11103_gb300 import fsp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIELDS = {
    "fsp_config": (fsp._Config, ["scheme", "precision", "interp", "ppm", "linear_weights", "bc", "gamma",
                                 "lf_alpha", "eps", "bc_state", "weights", "mid_split", "scheme_alpha"]),
    "fsp_block": (fsp._Block, ["ni", "nj", "ld", "period"]),
    "fsp_link": (fsp._Link, ["nbr", "face", "reversed", "offset"]),
    "fsp3_block": (fsp._Block3, ["ni", "nj", "nk", "bc", "period"]),
}


def test_struct_layouts_match_the_header(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc is needed")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "fsp.h"', "int main(void) {"]
    for st, (_, names) in FIELDS.items():
        lines.append(f'  printf("{st} sizeof %zu\\n", sizeof({st}));')
        for n in names:
            lines.append(f'  printf("{st} {n} %zu %zu\\n", offsetof({st}, {n}), sizeof((({st}*)0)->{n}));')
    lines += ["  return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c = {}
    for line in filter(None, out):
        parts = line.split()
        if parts[1] == "sizeof":
            c[(parts[0], None)] = int(parts[2])
        else:
            c[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    for st, (cls, names) in FIELDS.items():
        assert ctypes.sizeof(cls) == c[(st, None)], st
        for n in names:
            f = getattr(cls, n)
            assert (f.offset, f.size) == c[(st, n)], (st, n)
