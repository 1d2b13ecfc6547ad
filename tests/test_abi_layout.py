"""The ctypes structures of the Python binding have the C layout of include/sais.h: every
structure's size and every field's offset, as gcc lays them out, equal ctypes' (CPU only)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_2501_04971_gb300 import sais

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [sais.sais_problem_desc, sais.sais_problem_scalars, sais.sais_layout,
           sais.sais_sample_params, sais.sais_solve_params, sais.sais_tuning,
           sais.sais_solve_result, sais.sais_plan]


def _c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sais.h"', 'int main(void) {']
    for st in STRUCTS:
        name = st.__name__
        lines.append(f'  printf("%s size %zu\\n", "{name}", sizeof({name}));')
        for field, *_ in st._fields_:
            lines.append(f'  printf("%s %s %zu\\n", "{name}", "{field}", '
                         f'offsetof({name}, {field}));')
    lines += ['  return 0;', '}']
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                       check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        a, b, c = line.split()
        layout[(a, b)] = int(c)
    return layout


def test_binding_structs_match_the_header():
    layout = _c_layout()
    for st in STRUCTS:
        name = st.__name__
        assert ctypes.sizeof(st) == layout[(name, "size")], name
        for field, *_ in st._fields_:
            assert getattr(st, field).offset == layout[(name, field)], (name, field)
