"""CPU checks of the C ABI boundary: libsfft builds, loads without a GPU and exports every
function include/sfft.h declares; the package never reaches the CPU oracle."""
import ast
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sfft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfft_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("sfft_plan_create", "sfft_execute", "sfft_execute_batch", "sfft_submit",
                 "sfft_poll", "sfft_plan_destroy", "sfft_error_string"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2011_05749_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2011_05749_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.EXPORTS)


def test_error_strings_without_gpu():
    from paper_2011_05749_gb300 import _lib
    lib = _lib.load()
    assert lib.sfft_error_string(0) == b"ok"
    assert b"invalid" in lib.sfft_error_string(-1)


def test_product_code_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2011_05749_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            path = os.path.join(dirpath, fn)
            if fn.endswith(".py"):
                tree = ast.parse(open(path).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert not any(a.name.split(".")[0] == "oracle" for a in node.names), path
                    if isinstance(node, ast.ImportFrom):
                        assert (node.module or "").split(".")[0] != "oracle", path
            if fn.endswith((".cu", ".cuh", ".h", ".cpp")):
                assert "sfft_oracle" not in open(path).read(), path
