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
