"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/corutv.h declares (no compute calls: this runs without a GPU)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "corutv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"typedef[^;]*;", "", text)  # types (the callback) are not entry points
    return sorted(set(re.findall(r"\b(corutv_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1906_04572_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("corutv_create", "corutv_destroy", "corutv_factor", "corutv_rpca", "corutv_submit",
                     "corutv_poll"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1906_04572_gb300 import corutv
    assert sorted(corutv.EXPORTED) == _declared()


def test_create_fails_loudly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1906_04572_gb300 import corutv
    with pytest.raises(corutv.CorutvError) as ei:
        corutv.corutv_create(0)
    assert ei.value.status == corutv.ECUDA


def test_library_is_sm103a_only():
    from paper_1906_04572_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_structs_match_the_header(tmp_path):
    """corutv_opts and corutv_request as the C compiler lays them out (size and
    every field's offset, from a program built against include/corutv.h)
    equal the ctypes structures the binding passes across the boundary."""
    import shutil
    import subprocess
    from paper_1906_04572_gb300 import corutv
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"corutv_opts": corutv.Opts, "corutv_request": corutv.Request}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "corutv.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
