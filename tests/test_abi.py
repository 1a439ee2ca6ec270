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


def test_every_entry_point_checks_its_arguments_on_the_host():
    """Null handles, bad sizes and bad modes come back as errors from the
    host-side checks of each entry point, before any CUDA call."""
    from paper_1612_01855_gb300 import binding
    lib = binding.load_library()
    E = binding.TRSM_EINVAL
    p16 = ctypes.c_void_p(16)
    # solves on a null plan, under every schedule and workspace form
    for sched in (0, 1, 2, 3, 5):
        assert lib.trsm_solve_schedule(None, p16, 1, 8, p16, 8, sched, None) == E
    assert lib.trsm_plan_sliced(None, None) == E
    assert lib.trsm_residual_plan(None, p16, 1, 8, p16, 8, p16, 8, 7, p16, None) == E
    assert lib.trsm_solve_ws(None, p16, 1, 8, p16, 8, p16, 1 << 20, None) == E
    assert lib.trsm_solve_noalloc(None, p16, 1, 8, p16, 8, None) == E
    assert lib.trsm_plan_mixed(None, p16, 8, binding.TRSM_INNER_TF32, None) == E
    it = ctypes.c_int(7)
    up = ctypes.c_double(1.0)
    assert lib.trsm_solve_mixed(None, p16, 1, 8, p16, 8, 0, 10, 1e-12, ctypes.byref(it), ctypes.byref(up), None) == E
    assert it.value == 0 and up.value == 0.0
    # host-buffer entry
    assert lib.trsm_host(None, 8, 8, 4, p16, 1, 8, p16, 8, None) == E
    assert lib.trsm_host(p16, 0, 8, 4, p16, 1, 8, p16, 8, None) == E
    assert lib.trsm_host(p16, 8, 8, 4, None, 1, 8, p16, 8, None) == E
    assert lib.trsm_host(p16, 8, 8, 4, p16, -1, 8, p16, 8, None) == E
    # plan queries on a null plan
    assert lib.trsm_plan_device_bytes(None) == 0
    assert lib.trsm_plan_sizes(None, None, None, None) == E
    # batches: null handle
    item, row = ctypes.c_int(5), ctypes.c_int64(5)
    assert lib.trsm_batch_run(None, None) == E
    assert lib.trsm_batch_capture(None, None) == E
    assert lib.trsm_batch_launch_graph(None, None) == E
    assert lib.trsm_batch_status(None, None, ctypes.byref(item), ctypes.byref(row)) == E
    assert item.value == -1 and row.value == -1
    assert lib.trsm_batch_workspace_bytes(None) == 0
    lib.trsm_batch_destroy(None)
    # engine building blocks
    assert lib.trsm_tc_gemm_selftest(4, p16, p16, p16, 128, 128, 64, p16, None) == -1   # no mode 4
    assert lib.trsm_tc_gemm_selftest(0, p16, p16, p16, 128, 128, 60, p16, None) == -1   # K not a multiple of 8
    for planes in (4, 9):  # 5 to 8 planes
        assert lib.trsm_residual_sliced(p16, 8, 8, p16, 1, 8, p16, 8, p16, 8, planes, p16, None) == -1
    assert lib.trsm_residual_sliced(None, 8, 8, p16, 1, 8, p16, 8, p16, 8, 7, p16, None) == -1
    assert lib.trsm_wait_selftest(2, 1000, None) == E
    assert lib.trsm_wait_selftest(0, 0, None) == E


def test_workspace_pool_queries_without_gpu():
    """The pool queries need no device work: without a GPU the trim reports
    the missing device and nothing is reserved."""
    import torch
    from paper_1612_01855_gb300 import binding
    lib = binding.load_library()
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    assert lib.trsm_workspace_reserved_bytes() == 0
    assert lib.trsm_workspace_trim(0) == binding.TRSM_ECUDA


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
