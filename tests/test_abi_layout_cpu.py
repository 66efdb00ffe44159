"""The ctypes mirrors of the C-ABI structs match the header's layout.

A small C program, compiled with the host compiler against include/bembel.h, prints the
size of every struct and the offset of every field; the binding's ctypes structures must
give the same numbers (a field added to the header but not to the binding, or in another
order, would otherwise shift every later field silently)."""
import os
import shutil
import subprocess

import pytest

from paper_1906_00785_gb300 import capi

HERE = os.path.dirname(os.path.abspath(__file__))
INCLUDE = os.path.join(HERE, "..", "include")

STRUCTS = {
    "bembel_geom_desc": capi.GeomDesc,
    "bembel_opts": capi.Opts,
    "bembel_op_info": capi.OpInfo,
    "bembel_solve_opts": capi.SolveOpts,
    "bembel_solve_info": capi.SolveInfo,
    "bembel_tune_report": capi.TuneReport,
    "bembel_batch_item": capi.BatchItem,
}


def c_program():
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "bembel.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    return "\n".join(lines) + "\n"


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a host C compiler")
def test_struct_layouts_match(tmp_path):
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text(c_program())
    subprocess.run(["gcc", "-std=c11", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, key, val = line.split()
            got[(name, key)] = int(val)
    for cname, py in STRUCTS.items():
        assert got[(cname, "size")] == capi.C.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
