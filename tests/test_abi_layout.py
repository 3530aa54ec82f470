"""The ctypes mirrors of the ABI structs (paper_1707_05058_gb300/cdsdp.py) have
the layout of the C structs in include/cdsdp.h: same size, same field offsets.
A mismatch would let cdsdp_default_opts write past the Python buffer.  Host
only: a small C program compiled with the system C compiler reports the C side."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_layout(struct, fields, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cdsdp.h"', 'int main(void) {',
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ['  return 0;', '}']
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("name,struct", [("Opts", "cdsdp_opts"), ("Info", "cdsdp_info_t")])
def test_ctypes_struct_matches_c(lib, tmp_path, name, struct):
    py = getattr(lib, name)
    fields = [f for f, _ in py._fields_]
    size, offsets = _c_layout(struct, fields, tmp_path)
    assert ctypes.sizeof(py) == size
    assert [getattr(py, f).offset for f in fields] == offsets
