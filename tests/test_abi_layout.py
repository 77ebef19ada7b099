"""The ctypes structures of the binding match the C structures of
include/qtt.h field by field: sizes and offsets printed by a C program
compiled against the header (no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2512_07811_gb300 import qtt as Q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "qtt_round_info": Q.RoundInfo,
    "qtt_rve": Q.RVE,
    "ms_opts": Q.MSOpts,
    "ms_report": Q.MSReport,
    "qtt_cross_fn": Q.CrossFn,
    "qtt_cross_info": Q.CrossInfo,
    "qtt_amen_info": Q.AmenInfo,
}


def _probe(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "qtt.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    table = {}
    for line in out.splitlines():
        a, b, v = line.split()
        table[(a, b)] = int(v)
    return table


def test_struct_layouts_match_the_header(tmp_path):
    table = _probe(tmp_path)
    for cname, py in STRUCTS.items():
        assert table[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert table[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
