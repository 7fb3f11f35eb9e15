"""The ctypes structures of the Python binding against the C structures of
include/*.h (no GPU): a small C program, compiled here with the host
compiler, prints sizeof and offsetof of every field, and each must equal the
binding's.  A field added, dropped, reordered or retyped on one side only
fails here instead of corrupting calls silently."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2507_09435_gb300 import mpm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = [mpm.mpm_scene_desc, mpm.mpm_material, mpm.mpm_newton_report, mpm.mpm_step_report,
           mpm.mpm_request, mpm.mpm_request_result, mpm.mpm_server_stats]


def test_binding_structs_match_the_headers(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mpm_serve.h"', "int main(void) {"]
    for st in STRUCTS:
        name = st.__name__
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'  printf("{name} {field} %zu %zu\\n", offsetof({name}, {field}), '
                         f'sizeof((({name}*)0)->{field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c_layout = {}
    for ln in out:
        parts = ln.split()
        if len(parts) == 3:
            c_layout[(parts[0], "")] = (int(parts[2]),)
        elif len(parts) == 4:
            c_layout[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    for st in STRUCTS:
        name = st.__name__
        assert c_layout[(name, "")] == (ctypes.sizeof(st),), name
        for field, _ in st._fields_:
            desc = getattr(st, field)
            assert c_layout[(name, field)] == (desc.offset, desc.size), (name, field)
