"""The Python binding's ctypes structs have the C layout of include/stodip_op.h.

A small C program, compiled by the host compiler against the header, prints
offsetof and sizeof of every field the binding declares (by the header's
field names) and the size of each struct; the ctypes structs must match field
for field.  A renamed, reordered, resized or missing field fails here instead
of corrupting a call.  CPU only: nothing is executed on a GPU.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _structs():
    from paper_2408_02367_gb300 import op
    # C struct name -> (ctypes struct, {ctypes field name: C field name} where they differ)
    return {
        "sdp_plan_desc": (op.PlanDesc, {}),
        "sdp_tuning": (op.Tuning, {}),
        "sdp_work": (op.Work, {"in_": "in"}),
    }


def _c_layout(tmp_path, structs):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "stodip_op.h"', "int main(void) {"]
    for cname, (cls, rename) in structs.items():
        lines.append(f'    printf("{cname} . %zu 0\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            f = rename.get(fname, fname)
            lines.append(f'    printf("{cname} {fname} %zu %zu\\n", offsetof({cname}, {f}), '
                         f"sizeof((({cname}*)0)->{f}));")
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    layout = {}
    for line in out.splitlines():
        cname, fname, off, size = line.split()
        layout[(cname, fname)] = (int(off), int(size))
    return layout


def test_ctypes_structs_match_the_header(tmp_path):
    structs = _structs()
    layout = _c_layout(tmp_path, structs)
    for cname, (cls, _) in structs.items():
        assert ctypes.sizeof(cls) == layout[(cname, ".")][0], cname
        for fname, _ in cls._fields_:
            field = getattr(cls, fname)
            assert (field.offset, field.size) == layout[(cname, fname)], (cname, fname)
