"""The Python binding's ctypes structures match the C header's layout: for every public struct, its size and the
offset of every field, as gcc lays out include/tc.h on this machine (no GPU needed)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["tc_allocator", "tc_graph_info", "tc_tuning", "tc_server_config", "tc_request_result", "tc_prune_stats",
           "tc_unfused_stats", "tc_server_stats"]


def _c_layout():
    import paper_1909_02127_gb300 as tc
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tc.h"', 'int main(void) {']
    for name in STRUCTS:
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(tc, name)._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ['  return 0;', '}']
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, key, value = line.split()
        layout[(name, key)] = int(value)
    return layout


def test_ctypes_structures_match_the_header():
    import ctypes

    import paper_1909_02127_gb300 as tc
    layout = _c_layout()
    for name in STRUCTS:
        cls = getattr(tc, name)
        assert ctypes.sizeof(cls) == layout[(name, "size")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == layout[(name, field)], (name, field)
