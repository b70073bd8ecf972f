"""The ctypes mirrors of the C ABI structs (paper_1612_04846_gb300/bura.py) against include/bura.h.

A C program compiled here with the host compiler prints sizeof and offsetof of every field of every
struct the binding mirrors; ctypes must agree, or arguments would be read from the wrong bytes.
"""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_1612_04846_gb300 import bura

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"bura_grid": bura.bura_grid, "bura_options": bura.bura_options, "bura_stats": bura.bura_stats,
           "bura_kernel_prof": bura.bura_kernel_prof, "bura_server_options": bura.bura_server_options,
           "bura_request": bura.bura_request, "bura_request_info": bura.bura_request_info,
           "bura_server_stats": bura.bura_server_stats, "bura_csr": bura.bura_csr}


def test_struct_layouts_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bura.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    lines += ["return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for name, cls in STRUCTS.items():
        assert int(out[name + " size"]) == C.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(out[name + "." + fname]) == getattr(cls, fname).offset, (name, fname)
