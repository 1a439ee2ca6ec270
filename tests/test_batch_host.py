"""Host-side logic of the batch builder (no GPU: sizing and validation make
no CUDA call for items without a plan): argument checks and the workspace
each dtype lays out."""
import ctypes

import pytest


def _size(lib, binding, specs, dtype=0):
    """specs: (n, k, n0, tile_cols) per item; device pointers are never
    dereferenced while sizing, so placeholders stand in for them."""
    items = (binding.BatchItem * len(specs))()
    for i, (n, k, n0, tile) in enumerate(specs):
        it = items[i]
        it.L, it.ldl, it.plan = 0x10000 + 0x1000 * i, n, None
        it.B, it.ldb = 0x20000000 + 0x100000 * i, n
        it.X, it.ldx = 0x40000000 + 0x100000 * i, n
        it.n, it.k, it.n0, it.tile_cols = n, k, n0, tile
    out = ctypes.c_size_t(0)
    rc = lib.trsm_batch_workspace_size(items, len(specs), dtype, ctypes.byref(out))
    return rc, out.value


@pytest.fixture(scope="module")
def host_lib():
    from paper_1612_01855_gb300 import binding
    return binding.load_library(), binding


def test_batch_items_are_validated(host_lib):
    lib, binding = host_lib
    ok = (300, 40, 32, 0)
    assert _size(lib, binding, [ok])[0] == 0
    assert _size(lib, binding, [(300, 40, 48, 0)])[0] == binding.TRSM_EINVAL  # n0 only 32 or 64
    for tile in (5, 18, 36, -1):  # FP64 widths: 1 to 3 and multiples of 4 up to 32
        assert _size(lib, binding, [(300, 40, 32, tile)])[0] == binding.TRSM_EINVAL
    for tile in (1, 2, 3, 4, 12, 20, 24, 28):
        assert _size(lib, binding, [(300, 40, 32, tile)])[0] == 0
        assert _size(lib, binding, [(300, 40, 64, tile)], dtype=1)[0] == binding.TRSM_EINVAL  # FP32: 8, 16, 32
    assert _size(lib, binding, [(0, 40, 32, 0)])[0] == binding.TRSM_EINVAL
    assert _size(lib, binding, [(300, 0, 32, 0)])[0] == binding.TRSM_EINVAL
    assert _size(lib, binding, [ok], dtype=2)[0] == binding.TRSM_EINVAL
    assert _size(lib, binding, [])[0] == binding.TRSM_EINVAL


def test_batch_workspace_by_dtype(host_lib):
    """FP64 keeps a working copy of B (grows with k by at least 8 bytes per
    element); FP32 keeps only the inverted blocks and tables (independent of
    k).  Splitting k = 40 into 32 + 8 columns costs a part's tables and
    counters, not a second copy of the inverted blocks."""
    lib, binding = host_lib
    n = 300
    f64 = {k: _size(lib, binding, [(n, k, 32, 0)])[1] for k in (32, 40, 64)}
    assert f64[64] - f64[32] >= 8 * n * 32
    f32 = {k: _size(lib, binding, [(n, k, 64, 0)], dtype=1)[1] for k in (1, 40, 256)}
    assert len(set(f32.values())) == 1
    inv = 4 * 64 * 64 * ((n + 63) // 64)
    assert f32[1] >= inv
    split, whole = _size(lib, binding, [(n, 40, 32, 0)])[1], _size(lib, binding, [(n, 40, 32, 32)])[1]
    assert whole <= split < whole + 8 * 32 * 32 * ((n + 31) // 32)  # less than one more set of 32 x 32 blocks
