"""The ctypes mirrors of the C ABI's option and statistics structs (paper_2306_01098_gb300/hisq.py)
have the layout of include/hisq.h: a small C program compiled with gcc against the header
prints every field's offset and each struct's size, which must equal the ctypes ones.  A field
added, dropped or reordered on one side only fails here (no GPU needed)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {"hisq_opts": "Opts", "hisq_solve_opts": "SolveOpts", "hisq_stats": "Stats",
           "hisq_net_opts": "NetOpts", "hisq_peaks": "Peaks"}


def _c_layout(tmp_path, hisq):
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "hisq.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        cls = getattr(hisq, pyname)
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, key, value = line.split()
        out[(cname, key)] = int(value)
    return out


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ctypes_structs_match_the_header(tmp_path):
    import ctypes

    from paper_2306_01098_gb300 import hisq
    c = _c_layout(tmp_path, hisq)
    for cname, pyname in STRUCTS.items():
        cls = getattr(hisq, pyname)
        assert ctypes.sizeof(cls) == c[(cname, "size")], cname
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == c[(cname, field)], (cname, field)


def _header_fields():
    """field names of every `typedef struct { ... } name;` in include/hisq.h, in order"""
    src = open(os.path.join(ROOT, "include", "hisq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(hisq_\w+)\s*;", src, flags=re.S):
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            # "double lr, beta1, beta2, eps" -> every declarator; arrays keep their name
            head, _, rest = decl.partition(",")
            declarators = [head.split()[-1]] + [d.strip() for d in rest.split(",") if d.strip()] if rest else \
                [head.split()[-1]]
            names += [re.sub(r"\[.*\]", "", d).lstrip("*") for d in declarators]
        out[name] = names
    return out


def test_ctypes_structs_have_every_header_field():
    from paper_2306_01098_gb300 import hisq
    fields = _header_fields()
    for cname, pyname in STRUCTS.items():
        assert [f for f, _ in getattr(hisq, pyname)._fields_] == fields[cname], cname
