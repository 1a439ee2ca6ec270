"""Host-side checks of the C ABI (no GPU needed): the library builds, loads
and exports every function that include/*.h declares; the binding knows the
same names; the product and the oracle do not import each other."""
import glob
import os
import re
import ctypes

import pytest

from conftest import ROOT


def header_functions():
    names = []
    for path in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("defined",):
                names.append(name)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ("trsm_plan", "trsm_solve", "trtri_blocks", "trsm_destroy"):
        assert must in names


def test_library_builds_and_exports_every_symbol():
    from paper_1612_01855_gb300 import build as pkg_build
    from paper_1612_01855_gb300 import binding
    path = pkg_build.build()
    lib = ctypes.CDLL(path)
    for name in header_functions():
        assert hasattr(lib, name), f"{name} declared but not exported"
        assert name in binding.SIGNATURES, f"{name} has no binding"
    assert set(binding.SIGNATURES) <= set(header_functions())


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1612_01855_gb300 import binding
    with pytest.raises(ImportError):
        binding._lib = None
        try:
            binding.load_library(str(tmp_path / "missing.so"))
        finally:
            binding._lib = None


def test_error_strings_and_counters_without_gpu():
    from paper_1612_01855_gb300 import binding
    lib = binding.load_library()
    assert lib.trsm_error_string(0) == b"success"
    assert b"singular" in lib.trsm_error_string(-2) or b"diagonal" in lib.trsm_error_string(-2)
    assert lib.trsm_singular_index() == -1
    assert lib.trsm_launch_count(1) >= 0


def test_invalid_arguments_rejected_before_any_device_work():
    """Bad sizes are rejected on the host (no CUDA call is made)."""
    from paper_1612_01855_gb300 import binding
    lib = binding.load_library()
    h = ctypes.c_void_p()
    assert lib.trsm_plan(None, 4, 4, 2, None, ctypes.byref(h)) == binding.TRSM_EINVAL
    assert lib.trsm_plan(ctypes.c_void_p(16), 0, 4, 2, None, ctypes.byref(h)) == binding.TRSM_EINVAL
    assert lib.trsm_plan(ctypes.c_void_p(16), 8, 4, 2, None, ctypes.byref(h)) == binding.TRSM_EINVAL
    assert lib.trsm_plan(ctypes.c_void_p(16), 8, 8, 0, None, ctypes.byref(h)) == binding.TRSM_EINVAL
    assert lib.trtri_blocks(ctypes.c_void_p(16), 8, 8, 0, ctypes.c_void_p(16), None) == binding.TRSM_EINVAL
    assert lib.trsm_solve(None, None, 1, 1, None, 1, None) == binding.TRSM_EINVAL


def _imports(path):
    src = open(path).read()
    return re.findall(r"^\s*(?:from|import)\s+([\w\.]+)", src, flags=re.M)


def test_product_and_oracle_are_independent():
    for path in glob.glob(os.path.join(ROOT, "paper_1612_01855_gb300", "**", "*.py"), recursive=True):
        assert not any(m.split(".")[0] == "oracle" for m in _imports(path)), path
    for path in glob.glob(os.path.join(ROOT, "paper_1612_01855_gb300", "csrc", "*")):
        assert "oracle" not in open(path).read().lower().replace("oracle-free", ""), path
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert not any(m.startswith("paper_1612_01855_gb300") for m in _imports(path)), path
