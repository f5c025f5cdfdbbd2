"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/wam.h declares; the binding mirrors those names.  No
compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wam.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[a-z_]+\s+)*[a-z_]+\s*\*?\s*(wam_[a-z0-9_]+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1508_04458_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("wam_create", "wam_destroy", "wam_set_data", "wam_reconstruct", "wam_project",
                 "wam_backproject", "wam_haar", "wam_synthesize", "wam_forward",
                 "wam_split_backproject", "wam_z0", "wam_update", "wam_expand", "wam_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_mirrors_the_header(lib):
    from paper_1508_04458_gb300 import wam
    assert sorted(wam.EXPORTED) == declared_functions()


def test_struct_layouts_match_header():
    # field order and count of the ctypes mirrors follow the header text
    from paper_1508_04458_gb300 import wam
    src = open(HEADER).read()
    body = re.search(r"typedef struct \{(.*?)\} wam_geometry;", src, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"([a-z_0-9]+)\s*[,;]", body)
    assert [f for f, _ in wam.wam_geometry._fields_] == fields


def test_null_context_is_rejected_without_gpu(lib):
    # argument checks run before any CUDA call
    lib.wam_reconstruct.restype = ctypes.c_int
    assert lib.wam_reconstruct(None, None, None, None, None, 0, None) == -1
    lib.wam_create.restype = ctypes.c_int
    out = ctypes.c_void_p()
    assert lib.wam_create(None, ctypes.byref(out)) == -1


def test_every_binding_call_passes_the_declared_argument_count():
    # each call of a C-ABI function in the tests, the benchmark and the
    # package passes as many arguments as its ctypes prototype (the header's)
    import ast
    import glob
    from paper_1508_04458_gb300 import wam
    files = glob.glob(os.path.join(ROOT, "tests", "*.py")) + [os.path.join(ROOT, "bench.py")] + \
        glob.glob(os.path.join(ROOT, "paper_1508_04458_gb300", "*.py"))
    bad = []
    for f in files:
        for node in ast.walk(ast.parse(open(f).read())):
            if isinstance(node, ast.Call) and isinstance(node.func, ast.Attribute) and node.func.attr in wam._PROTOS:
                if any(isinstance(a, ast.Starred) for a in node.args):
                    continue
                if len(node.args) != len(wam._PROTOS[node.func.attr][1]):
                    bad.append((os.path.basename(f), node.lineno, node.func.attr))
    assert not bad, bad
