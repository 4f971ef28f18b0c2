"""The Python binding's ctypes mirrors of include/gcdf.h agree with the C
compiler's view of the header: every struct's size and every field's offset,
and every enum constant.  A plain C program built with the host compiler
prints them (no GPU, no CUDA headers: the header is plain C)."""
import ctypes
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {"NetDesc": "gcdf_net_desc", "FitDesc": "gcdf_fit_desc", "PlanParams": "gcdf_plan_params",
           "PlanProblem": "gcdf_plan_problem", "ServerDesc": "gcdf_server_desc",
           "PlanRequest": "gcdf_plan_request", "PlanResult": "gcdf_plan_result",
           "ServerStats": "gcdf_server_stats"}


def _c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_2601_18548_gb300 import _lib
    hdr = open(os.path.join(ROOT, "include", "gcdf.h")).read()
    enums = sorted(set(re.findall(r"\b(GCDF_[A-Z0-9_]+)\s*=", hdr)))
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gcdf.h"', "int main(void) {"]
    for py, c in STRUCTS.items():
        lines.append(f'  printf("S {py} %zu\\n", sizeof({c}));')
        for name, _ in getattr(_lib, py)._fields_:
            lines.append(f'  printf("F {py} {name} %zu\\n", offsetof({c}, {name}));')
    for e in enums:
        lines.append(f'  printf("E {e} %d\\n", (int){e});')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return out.split("\n"), enums


def test_structs_and_enums_match_the_header():
    from paper_2601_18548_gb300 import _lib
    lines, enums = _c_layout()
    seen = 0
    for ln in lines:
        parts = ln.split()
        if not parts:
            continue
        if parts[0] == "S":
            assert ctypes.sizeof(getattr(_lib, parts[1])) == int(parts[2]), ln
        elif parts[0] == "F":
            assert getattr(getattr(_lib, parts[1]), parts[2]).offset == int(parts[3]), ln
        elif parts[0] == "E":
            assert getattr(_lib, parts[1]) == int(parts[2]), ln
        seen += 1
    assert seen == len(STRUCTS) + sum(len(getattr(_lib, p)._fields_) for p in STRUCTS) + len(enums)
