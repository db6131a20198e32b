"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/tvs.h declares; the Python binding declares the same set.
No compute call is made here."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tvs.h")


def _declared_functions(path):
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s+\**\s*([A-Za-z_]\w*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "return")))


@pytest.fixture(scope="module")
def built_lib():
    import __graft_entry__ as g
    return g._build_module().build()


def test_header_declares_expected_api():
    names = _declared_functions(HEADER)
    for must in ("tv_prox", "pgd_solve", "proxskip_solve", "pdhg_solve", "pdhgskip_solve",
                 "fista_solve", "tvs_create", "tvs_problem_create", "tvs_coin"):
        assert must in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in _declared_functions(HEADER) if not hasattr(lib, n)]
    assert not missing, f"missing exports: {missing}"


def test_binding_declares_the_header_api(built_lib):
    from paper_2411_00688_gb300 import _lib
    bound = sorted(n for n, _, _ in _lib.SIGNATURES)
    assert bound == _declared_functions(HEADER)


def test_struct_layout_matches_c(tmp_path, built_lib):
    """ctypes mirrors of the header structs have the sizes and field offsets a C
    compiler gives the header's structs."""
    import shutil
    import subprocess
    from paper_2411_00688_gb300 import _lib as L
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"tvs_op_desc": L.OpDesc, "tvs_problem_desc": L.ProblemDesc,
               "tvs_fb_params": L.FBParams, "tvs_pd_params": L.PDParams, "tvs_trace": L.Trace,
               "tvs_rof_params": L.RofParams, "tvs_pdx_params": L.PDXParams}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tvs.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


@pytest.mark.parametrize("dims,ndim,warm_too", [((1 << 30, 1 << 30, 1), 2, True),
                                                ((1 << 30, 1 << 30, 1 << 30), 3, True),
                                                ((1 << 16, 1 << 16, 1 << 16), 3, True),
                                                ((1024, 1366, 1), 2, True),
                                                ((1025, 1024, 1), 2, False)])
def test_noalloc_rejects_oversized_requests_before_any_cuda_call(built_lib, dims, ndim, warm_too):
    """Sizes whose scratch would exceed the static array -- including products of
    the sides that wrap around 64 bits -- are refused with TVS_EUNSUPPORTED by
    arithmetic alone: the call returns before touching CUDA (this machine has no
    GPU), so nothing can have been launched.  The pointers are never dereferenced.
    A cold start needs four FP32 dual planes per axis (1025 x 1024 is over the
    32 MiB limit), a caller-owned dual three (1024 x 1366 is over it)."""
    lib = ctypes.CDLL(built_lib)
    fn = lib.tv_prox_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                   ctypes.c_void_p]
    d = (ctypes.c_int * 3)(*dims)
    assert fn(ndim, d, ctypes.c_void_p(256), ctypes.c_void_p(512), 0.1, 5, 0, None, 0, None) == 6
    if warm_too:
        assert fn(ndim, d, ctypes.c_void_p(256), ctypes.c_void_p(512), 0.1, 5, 0, ctypes.c_void_p(1024), 0,
                  None) == 6
