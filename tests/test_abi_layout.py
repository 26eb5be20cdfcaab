"""The ctypes mirrors of the binding match the C structs of include/srw.h field
for field: a small C program compiled against the header prints each struct's
size and every field's offset, which must equal the ctypes layout."""

import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2607_00488_gb300 import srw as binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C struct name -> ctypes mirror (ctypes names a field "lambda_" where C says "lambda")
MIRRORS = {
    "srw_binning": binding._Binning,
    "srw_source": binding._Source,
    "srw_options": binding._Options,
    "srw_joint_response": binding._JointResponse,
    "srw_info_t": binding._Info,
    "srw_fit_opts": binding._FitOpts,
    "srw_scan_opts": binding._ScanOpts,
    "srw_scan_result": binding._ScanResult,
}


def _c_name(field):
    return field[:-1] if field.endswith("_") else field


def test_struct_layouts_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include "srw.h"', "#include <stdio.h>", "#include <stddef.h>", "int main(void) {"]
    for cname, mirror in MIRRORS.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in mirror._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f[0], cname, _c_name(f[0])))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            s, f, v = ln.split()
            got[(s, f)] = int(v)
    for cname, mirror in MIRRORS.items():
        assert got[(cname, "size")] == ctypes.sizeof(mirror), cname
        for f in mirror._fields_:
            assert got[(cname, f[0])] == getattr(mirror, f[0]).offset, (cname, f[0])
