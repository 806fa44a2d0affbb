"""The ctypes structures of the binding and the record dtype have the layout
of the C structures in include/epfft.h: a C program compiled with the host
compiler against the header prints every field offset and struct size."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_0802_2488_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RENAME = {"lambda_": "lambda"}  # Python keyword
PAIRS = [("epfft_options", B._Options), ("epfft_problem", B._Problem), ("epfft_path", B._Path),
         ("epfft_stats", B._Stats), ("epfft_serve_options", B._ServeOptions), ("epfft_fields", B._Fields)]


def c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "epfft.h"', "int main(void) {"]
    for cname, cls in PAIRS:
        lines.append(f'  printf("{cname} SIZE %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            g = RENAME.get(f, f)
            lines.append(f'  printf("{cname} {g} %zu\\n", offsetof({cname}, {g}));')
    lines.append('  printf("epfft_record SIZE %zu\\n", sizeof(epfft_record));')
    for f in B.RECORD_DTYPE.names:
        lines.append(f'  printf("epfft_record {f} %zu\\n", offsetof(epfft_record, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {(s, f): int(v) for s, f, v in (l.split() for l in out.splitlines())}


def test_struct_layouts_match_the_header(tmp_path):
    lay = c_layout(tmp_path)
    for cname, cls in PAIRS:
        assert lay[(cname, "SIZE")] == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert lay[(cname, RENAME.get(f, f))] == getattr(cls, f).offset, (cname, f)
    assert lay[("epfft_record", "SIZE")] == B.RECORD_DTYPE.itemsize
    for f in B.RECORD_DTYPE.names:
        assert lay[("epfft_record", f)] == B.RECORD_DTYPE.fields[f][1], f
