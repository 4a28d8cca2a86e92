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


def _c_kind(t):
    t = t.strip()
    if "*" in t:
        return "ptr"
    t = re.sub(r"\bconst\b", "", t).split()[0]
    return {"double": "f64", "uint64_t": "u64", "size_t": "u64", "int64_t": "i64", "lsq_ticket": "i64",
            "int32_t": "i32", "int": "i32", "lsq_status": "i32"}[t]


def _py_kind(ct):
    if ct is None:
        return "i32"  # ctypes' default return type
    if ct in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(ct, "_type_") and isinstance(ct._type_, type):
        return "ptr"
    size, signed = ctypes.sizeof(ct), ct(-1).value == -1 if ct is not ctypes.c_double else None
    if ct is ctypes.c_double:
        return "f64"
    return {(8, True): "i64", (8, False): "u64", (4, True): "i32", (4, False): "u32"}[(size, signed)]


def _prototypes():
    src = open(os.path.join(ROOT, "include", "lsq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for ret, name, args in re.findall(r"^([A-Za-z_][\w ]*?\**)\s*\b(lsq_[a-z_0-9]+)\(([^)]*)\);", src, flags=re.M):
        params = [a for a in (p.strip() for p in args.split(",")) if a and a != "void"]
        # drop the parameter name: everything up to the last identifier
        kinds = [_c_kind(re.sub(r"\b\w+$", "", p) if not p.endswith("*") else p) for p in params]
        out[name] = (_c_kind(ret), kinds)
    return out


def test_binding_argtypes_match_the_prototypes(libpath):
    """Every entry point the binding calls is declared to ctypes with the
    header's parameter kinds (pointer, 32/64-bit integer, double), so no
    argument is truncated or passed in the wrong register."""
    import paper_2506_03070_gb300 as P
    L = P.load(libpath)
    protos = _prototypes()
    assert set(protos) == set(_declared())
    for name, (ret, kinds) in protos.items():
        fn = getattr(L, name)
        assert fn.argtypes is not None, f"{name}: no argtypes in the binding"
        assert [_py_kind(a) for a in fn.argtypes] == kinds, name
        assert _py_kind(fn.restype) == ret, name
