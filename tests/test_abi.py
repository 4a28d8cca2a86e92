"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/lsq.h; the binding refuses to run without the library or
a GPU (no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lsq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsq_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2506_03070_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lsq_create", "lsq_destroy", "lsq_sketch", "lsq_sketch_indices", "lsq_precond", "lsq_lsqr",
                     "lsq_solve", "lsq_check", "lsq_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings_without_gpu(libpath):
    import paper_2506_03070_gb300 as P
    L = P.load(libpath)
    assert L.lsq_status_string(0) == b"LSQ_OK"
    assert L.lsq_status_string(-8) == b"LSQ_ERR_TIMEOUT"
    assert L.lsq_last_error(None) == b"null context"


def test_create_fails_loudly_without_gpu(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2506_03070_gb300 as P
    with pytest.raises(P.LsqError):
        P.Context(0)
