"""The binding's ctypes structures have the C layout of include/femamg.h: a small C program
compiled against the header prints sizeof and offsetof of every field, and each ctypes
Structure must agree field by field (a mismatch would hand the library shifted arguments
without any error)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C typedef name -> binding class name
PAIRS = {
    "fem_kuhn_desc": "KuhnDesc",
    "fem_target": "Target",
    "fem_assemble_opts": "AssembleOpts",
    "fem_system_info": "SystemInfo",
    "amg_opts": "AmgOpts",
    "amg_hier_info": "HierInfo",
    "pcg_opts": "PcgOpts",
    "pcg_result": "PcgResult",
    "fem_mesh_desc": "MeshDesc",
    "fem_errors_result": "ErrorsResult",
    "fem_mesh_info": "MeshInfo",
    "fem_refine_stats": "RefineStats",
    "bddc_opts": "BddcOpts",
}


def _c_layout(tmp_path, binding):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "femamg.h"', "int main(void) {"]
    for cname, pyname in PAIRS.items():
        cls = getattr(binding, pyname)
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));'
                         % (cname, fname, cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o",
                           str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True)
    got = {}
    for ln in out.splitlines():
        a, b, v = ln.split()
        got[(a, b)] = int(v)
    return got


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ctypes_structures_match_the_c_header(tmp_path):
    from paper_2102_03515_gb300 import _binding as B
    c = _c_layout(tmp_path, B)
    for cname, pyname in PAIRS.items():
        cls = getattr(B, pyname)
        assert C.sizeof(cls) == c[(cname, "size")], cname
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == c[(cname, fname)], (cname, fname)
