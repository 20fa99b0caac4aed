"""The C-ABI library builds, loads and exports every entry point of include/lcs.h.

No compute calls are made (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lcs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lcs_[a-z_]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    syms = declared_symbols()
    for s in ("lcs_init", "lcs_step", "lcs_migrate", "lcs_sort", "lcs_backward"):
        assert s in syms


def test_library_builds_and_exports_every_declared_symbol():
    import paper_2604_11008_gb300 as lcs
    from paper_2604_11008_gb300 import build
    build.build()
    L = lcs.lib()
    for s in declared_symbols():
        assert hasattr(L, s), s
    assert sorted(lcs.EXPORTS) == declared_symbols()


def test_binding_refuses_to_run_without_the_library(tmp_path, monkeypatch):
    import paper_2604_11008_gb300 as lcs
    monkeypatch.setattr(lcs, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(lcs, "_lib", None)
    with pytest.raises(ImportError):
        lcs.lib()


def test_binding_does_not_import_the_oracle():
    import ast
    pkg = os.path.join(ROOT, "paper_2604_11008_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                tree = ast.parse(open(os.path.join(dirpath, f)).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert all(not a.name.startswith("oracle") for a in node.names), f
                    if isinstance(node, ast.ImportFrom):
                        assert not (node.module or "").startswith("oracle"), f


def test_null_context_and_bad_arguments_are_rejected_without_gpu_work():
    import ctypes as C
    import paper_2604_11008_gb300 as lcs
    L = lcs.lib()
    assert L.lcs_init(None, 1, None, C.byref(C.c_void_p())) == lcs.LCS_ERR_ARG
    assert L.lcs_step(None, 1) == lcs.LCS_ERR_ARG
    assert L.lcs_sync(None) == lcs.LCS_ERR_ARG
    assert isinstance(L.lcs_last_error(None), bytes)
    L.lcs_destroy(None)
    assert L.lcs_partition(None, -1, 4, None, None, None, None) == lcs.LCS_ERR_ARG


def test_header_is_plain_c():
    """include/lcs.h compiles as C11 (no C++ or torch types in the ABI): the
    C example that the GPU tests build and run is checked for syntax here."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    from paper_2604_11008_gb300 import build
    cuda = os.path.dirname(os.path.dirname(build.nvcc()))
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-fsyntax-only",
                    os.path.join(ROOT, "tests", "c_abi", "uniform_flow.c"),
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include")],
                   check=True)
