"""The Python binding's structures match include/dirac.h byte for byte.

A small C program compiled with gcc against the header prints the size and
every member's offset of dirac_fields, dirac_plan and dirac_check_report;
the ctypes structures of paper_1309_3452_gb300/dirac.py must agree.  Runs on
the CPU (no device call).
"""
import ctypes as C
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def D():
    from paper_1309_3452_gb300 import build as B
    B.build()
    from paper_1309_3452_gb300 import dirac
    return dirac


def c_layout(tmp_path, struct, members):
    src = tmp_path / f"{struct}.c"
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dirac.h"', "int main(void) {",
             f'  printf("size %zu\\n", sizeof({struct}));']
    for m in members:
        lines.append(f'  printf("{m} %zu\\n", offsetof({struct}, {m}));')
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / struct
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


@pytest.mark.parametrize("struct,pyname", [("dirac_fields", "Fields"), ("dirac_plan", "Plan"),
                                           ("dirac_check_report", "CheckReport")])
def test_struct_layout_matches_header(D, tmp_path, struct, pyname):
    cls = getattr(D, pyname)
    members = [name for name, _ in cls._fields_]
    got = c_layout(tmp_path, struct, members)
    assert got["size"] == C.sizeof(cls)
    for name in members:
        assert got[name] == getattr(cls, name).offset, name
