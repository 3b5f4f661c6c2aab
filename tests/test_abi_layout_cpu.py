"""The Python binding's ctypes structures have the C header's layout: a small
C program built with gcc against include/polyclean.h prints the size and
every field offset of each public struct, and they must equal ctypes' own
(a field added on one side only would shift every later field)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_name(py_name):
    """C field name of a ctypes field (a trailing _ avoids a Python keyword)."""
    return py_name[:-1] if py_name.endswith("_") else py_name


STRUCTS = ["pc_plan_opts", "pc_plan_tuning", "pc_solve_opts", "pc_iter_record", "pc_solve_stats",
           "pc_dictionary", "pc_server_opts", "pc_job_times", "pc_kernel_time"]


def _c_layout(tmp_path):
    from paper_2406_01342_gb300 import abi
    lines = ["#include <stdio.h>", "#include <stddef.h>", "#include \"polyclean.h\"", "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for name, _ in getattr(abi, s)._fields_:
            lines.append(f'  printf("{s} {name} %zu\\n", offsetof({s}, {_c_name(name)}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ctypes_structs_match_the_header(tmp_path):
    from paper_2406_01342_gb300 import abi
    c = _c_layout(tmp_path)
    for s in STRUCTS:
        cls = getattr(abi, s)
        assert c[(s, "size")] == ctypes.sizeof(cls), s
        for name, _ in cls._fields_:
            assert c[(s, name)] == getattr(cls, name).offset, (s, name)
