"""CPU-side checks of the boundary: the library builds, loads and exports every
function include/gb300bfs.h declares; the binding wraps exactly those; the
product package never reaches the oracle and fails loudly without its CUDA
library.  No compute call is made (there is no GPU here)."""
import ast
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gb300bfs.h")
PKG = os.path.join(ROOT, "paper_2012_13548_gb300")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    names = set()
    for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s*([A-Za-z_]\w*)\s*\(", text, re.M):
        names.add(m.group(1))
    return names - {"if", "while", "for", "return", "sizeof"}


@pytest.fixture(scope="module")
def built_lib():
    from paper_2012_13548_gb300 import build_ext
    path = build_ext.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["kron_generate", "graph_build_csr", "bfs", "bfs_batch", "bfs_multi_graph",
                 "server_create", "server_submit", "server_poll", "gb_last_error"]:
        assert must in names, must


def test_library_exports_every_declared_symbol(built_lib):
    for name in sorted(declared_functions()):
        assert hasattr(built_lib, name), "missing export %s" % name


def test_binding_wraps_exactly_the_header(built_lib):
    from paper_2012_13548_gb300 import binding
    assert set(binding.exported_symbols()) == declared_functions()
    binding.lib()  # every signature resolves against the built library


def test_abi_version_call_needs_no_gpu(built_lib):
    built_lib.gb_abi_version.restype = ctypes.c_int
    assert built_lib.gb_abi_version() == 1
    built_lib.gb_last_error.restype = ctypes.c_char_p
    assert built_lib.gb_last_error() == b""


def test_product_package_never_imports_the_oracle():
    for fn in os.listdir(PKG):
        if not fn.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(PKG, fn)).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert not any(a.name.split(".")[0] == "oracle" for a in node.names), fn
            if isinstance(node, ast.ImportFrom):
                assert (node.module or "").split(".")[0] != "oracle", fn
    for fn in os.listdir(os.path.join(PKG, "csrc")):
        src = open(os.path.join(PKG, "csrc", fn)).read()
        assert "graph500_oracle" not in src and "gbo_" not in src, fn


def test_oracle_shares_no_code_with_the_library():
    src = open(os.path.join(ROOT, "oracle", "graph500_oracle.c")).read()
    assert "#include \"" not in src          # only system headers
    assert "gb300bfs" not in src


def test_missing_library_fails_loudly(monkeypatch):
    from paper_2012_13548_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "lib.so"))
    with pytest.raises(RuntimeError, match="missing"):
        binding.lib()
