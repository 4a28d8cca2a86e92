"""The Python binding's ctypes structures and constants against the C header
(no GPU): a C program compiled from include/lsq.h prints every struct's size
and field offsets and the values of the status, flag, precision, memory and
QR-mode constants; the binding must agree on all of them, or a call would
read its arguments from the wrong place."""
import ctypes
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {  # C typedef -> binding class name
    "lsq_problem": "Problem",
    "lsq_opts": "Opts",
    "lsq_info": "Info",
    "lsq_csr_problem": "CsrProblem",
    "lsq_batch_item": "BatchItem",
    "lsq_batch_result": "BatchResult",
    "lsq_serve_stats": "ServeStats",
}
CONSTANTS = {  # C macro or enumerator -> binding name
    "LSQ_OK": "LSQ_OK", "LSQ_PENDING": "LSQ_PENDING", "LSQ_ERR_ARG": "LSQ_ERR_ARG",
    "LSQ_ERR_NOCONV": "LSQ_ERR_NOCONV", "LSQ_ERR_TIMEOUT": "LSQ_ERR_TIMEOUT", "LSQ_ERR_ACCURACY": "LSQ_ERR_ACCURACY",
    "LSQ_PREC_FP64": "PREC_FP64", "LSQ_PREC_MIXED": "PREC_MIXED",
    "LSQ_MEM_DEVICE": "MEM_DEVICE", "LSQ_MEM_HOST": "MEM_HOST",
    "LSQ_FLAG_TIMING": "FLAG_TIMING", "LSQ_FLAG_NO_CHECK": "FLAG_NO_CHECK",
    "LSQ_FLAG_NATIVE_FP64": "FLAG_NATIVE_FP64", "LSQ_FLAG_NO_IMAGE": "FLAG_NO_IMAGE",
    "LSQ_FLAG_NO_FALLBACK": "FLAG_NO_FALLBACK", "LSQ_FLAG_AUTOTUNE": "FLAG_AUTOTUNE", "LSQ_FLAG_HBM": "FLAG_HBM",
    "LSQ_QR_AUTO": "QR_AUTO", "LSQ_QR_UNBLOCKED": "QR_UNBLOCKED", "LSQ_QR_BLOCKED": "QR_BLOCKED",
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    import paper_2506_03070_gb300 as P
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lsq.h"', "int main(void) {",
             '  printf("{\\"structs\\": {");']
    for k, (cname, pyname) in enumerate(STRUCTS.items()):
        fields = [f for f, _ in getattr(P, pyname)._fields_]
        parts = " ".join(f'printf("\\"{f}\\": %zu,", offsetof({cname}, {f}));' for f in fields)
        sep = "," if k + 1 < len(STRUCTS) else ""
        lines.append(f'  printf("\\"{cname}\\": {{"); {parts} printf("\\"__size\\": %zu}}{sep}", sizeof({cname}));')
    lines.append('  printf("}, \\"constants\\": {");')
    for k, cname in enumerate(CONSTANTS):
        sep = "," if k + 1 < len(CONSTANTS) else ""
        lines.append(f'  printf("\\"{cname}\\": %ld{sep}", (long)({cname}));')
    lines += ['  printf("}}\\n");', "  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    return json.loads(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)


@pytest.mark.parametrize("cname", list(STRUCTS))
def test_struct_layout_matches_header(c_layout, cname):
    import paper_2506_03070_gb300 as P
    cls = getattr(P, STRUCTS[cname])
    c = c_layout["structs"][cname]
    assert ctypes.sizeof(cls) == c["__size"], cname
    for f, _ in cls._fields_:
        assert getattr(cls, f).offset == c[f], (cname, f)


def test_constants_match_header(c_layout):
    import paper_2506_03070_gb300 as P
    for cname, pyname in CONSTANTS.items():
        assert getattr(P, pyname) == c_layout["constants"][cname], cname
