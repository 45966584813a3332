"""The Python binding's ctypes structures against the C declarations of
include/lbm.h: a small C program, compiled with the host compiler against the
header, prints every public structure's size and the offset of each field, and
the binding must agree field by field (a field added on one side only would
otherwise shift the rest silently)."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_1906_04722_gb300 as lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["lbm_params", "lbm_measurement", "lbm_increment", "lbm_schedule", "lbm_throat_result",
           "lbm_throat_surrogate_config", "lbm_tune_result", "lbm_surrogate_config"]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lbm.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(lbm, name)
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, field, value = line.split()
        layout[(name, field)] = int(value)
    return layout


def test_ctypes_structures_match_the_header(tmp_path):
    layout = _c_layout(tmp_path)
    for name in STRUCTS:
        cls = getattr(lbm, name)
        assert ctypes.sizeof(cls) == layout[(name, "size")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == layout[(name, field)], (name, field)
