"""The ctypes structures of the binding have the C header's layout: a small
C program compiled against include/emt.h prints sizeof and offsetof of every
field the binding declares, and both must agree (no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {"emt_options": "Options", "emt_material": "Material", "emt_physics": "Physics",
           "emt_layer": "Layer", "emt_world": "World", "emt_primaries": "Primaries",
           "emt_serve_options": "ServeOptions", "emt_step_record": "StepRecord", "emt_run_stats": "RunStats"}


def test_ctypes_structures_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2203_09467_gb300 import emt
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "emt.h"', "int main(void) {"]
    expect = []
    for cname, pyname in STRUCTS.items():
        cls = getattr(emt, pyname)
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(cls))
        for field, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {field}));')
            expect.append(getattr(cls, field).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == expect
