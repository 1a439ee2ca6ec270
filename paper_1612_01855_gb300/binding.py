"""Python binding of the C ABI in ``include/trsm_gb300.h``.

Argument marshalling only: every step of the method runs in the CUDA
library ``_build/libtrsm_gb300.so``.  There is no CPU fallback — if the
library is missing or no GPU is present, every call raises.

Matrices are torch tensors on a CUDA device, float64, in column-major layout
(``t.stride(0) == 1``; ``colmajor`` converts).  A tensor ``t`` of shape
(rows, cols) with strides (1, ld) is passed as pointer + leading dimension.
Work is enqueued on the current torch stream of the tensors' device.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtrsm_gb300.so")

TRSM_SUCCESS = 0
TRSM_EINVAL = -1
TRSM_ESINGULAR = -2
TRSM_ENOMEM = -3
TRSM_ECUDA = -4
TRSM_ETIMEOUT = -5
TRSM_ENOSCRATCH = -6
TRSM_ENOCONV = -7
TRSM_INNER_BF16 = 1
TRSM_INNER_TF32 = 2
TRSM_INNER_BF16X3 = 3
TRSM_INNER_FP16X3 = 4
TRSM_RESIDUAL_SLICED = 0
TRSM_RESIDUAL_FP64 = 1
TRSM_RESIDUAL_SLICED8 = 2
TRSM_RESIDUAL_ADAPTIVE = 3
TRSM_RESIDUAL_PROGRESSIVE = 4
TRSM_SOLVE_S_FP32 = 0x100
TRSM_SOLVE_S_TC = 0x200
TRSM_SOLVE_S_TC2 = 0x400
TRSM_SOLVE_S_TC1 = 0x800

TRSM_F64 = 0
TRSM_F32 = 1


class BatchItem(ctypes.Structure):
    """Mirror of trsm_batch_item (include/trsm_gb300.h)."""
    _fields_ = [("L", ctypes.c_void_p), ("ldl", ctypes.c_int64), ("plan", ctypes.c_void_p),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("X", ctypes.c_void_p),
                ("ldx", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("n0", ctypes.c_int64), ("tile_cols", ctypes.c_int64)]


# Every symbol the header declares, with (restype, argtypes).
_i64, _vp, _dp, _int = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int
_pi64 = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "trsm_plan": (_int, [_dp, _i64, _i64, _i64, _vp, ctypes.POINTER(_vp)]),
    "trsm_solve": (_int, [_vp, _dp, _i64, _i64, _dp, _i64, _vp]),
    "trsm_solve_schedule": (_int, [_vp, _dp, _i64, _i64, _dp, _i64, _int, _vp]),
    "trsm_solve_workspace_size": (_int, [_vp, _i64, ctypes.POINTER(ctypes.c_size_t)]),
    "trsm_solve_ws": (_int, [_vp, _dp, _i64, _i64, _dp, _i64, _vp, ctypes.c_size_t, _vp]),
    "trsm_solve_noalloc": (_int, [_vp, _dp, _i64, _i64, _dp, _i64, _vp]),
    "trsm_plan_sliced": (_int, [_vp, _vp]),
    "trsm_plan_mixed": (_int, [_vp, _dp, _i64, _int, _vp]),
    "trsm_solve_mixed": (_int, [_vp, _dp, _i64, _i64, _dp, _i64, _int, _int, ctypes.c_double,
                                ctypes.POINTER(_int), ctypes.POINTER(ctypes.c_double), _vp]),
    "trsm_batch_create": (_int, [ctypes.POINTER(BatchItem), _int, _int, ctypes.POINTER(_vp)]),
    "trsm_batch_workspace_size": (_int, [ctypes.POINTER(BatchItem), _int, _int, ctypes.POINTER(ctypes.c_size_t)]),
    "trsm_batch_create_ws": (_int, [ctypes.POINTER(BatchItem), _int, _int, _vp, ctypes.c_size_t, _vp,
                                    ctypes.POINTER(_vp)]),
    "trsm_batch_run": (_int, [_vp, _vp]),
    "trsm_batch_capture": (_int, [_vp, _vp]),
    "trsm_batch_launch_graph": (_int, [_vp, _vp]),
    "trsm_batch_status": (_int, [_vp, _vp, ctypes.POINTER(_int), ctypes.POINTER(ctypes.c_int64)]),
    "trsm_batch_destroy": (None, [_vp]),
    "trsm_batch_workspace_bytes": (ctypes.c_size_t, [_vp]),
    "trsm_host": (_int, [_dp, _i64, _i64, _i64, _dp, _i64, _i64, _dp, _i64, _vp]),
    "trtri_blocks": (_int, [_dp, _i64, _i64, _i64, _dp, _vp]),
    "trsm_destroy": (None, [_vp]),
    "trsm_plan_sizes": (_int, [_vp, _pi64, _pi64, _pi64]),
    "trsm_plan_device_bytes": (ctypes.c_size_t, [_vp]),
    "trsm_workspace_trim": (_int, [ctypes.c_size_t]),
    "trsm_workspace_reserved_bytes": (ctypes.c_size_t, []),
    "trsm_plan_lt": (_vp, [_vp, _pi64]),
    "trsm_sync_status": (_int, [_vp, _vp]),
    "trsm_singular_index": (_i64, []),
    "trsm_last_cuda": (_int, []),
    "trsm_error_string": (ctypes.c_char_p, [_int]),
    "trsm_launch_count": (_i64, [_int]),
    "trsm_fp64_peak": (_int, [_int, ctypes.POINTER(ctypes.c_double), _vp]),
    "trsm_fp32_peak": (_int, [_int, ctypes.POINTER(ctypes.c_double), _vp]),
    "trsm_tc_gemm_selftest": (_int, [_int, _vp, _vp, _vp, _i64, _i64, _i64, _vp, _vp]),
    "trsm_wait_selftest": (_int, [_int, _i64, _vp]),
    "trsm_residual_sliced": (_int, [_dp, _i64, _i64, _dp, _i64, _i64, _dp, _i64, _dp, _i64, _int, _vp, _vp]),
    "trsm_residual_plan": (_int, [_vp, _dp, _i64, _i64, _dp, _i64, _dp, _i64, _int, _vp, _vp]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class TrsmError(RuntimeError):
    def __init__(self, code, what):
        lib = load_library()
        msg = lib.trsm_error_string(code).decode()
        extra = ""
        if code == TRSM_ESINGULAR:
            extra = f" (row {lib.trsm_singular_index()})"
        elif code == TRSM_ECUDA:
            extra = f" (cudaError {lib.trsm_last_cuda()})"
        super().__init__(f"{what}: {msg}{extra} [{code}]")
        self.code = code


def _check(code, what):
    if code != TRSM_SUCCESS:
        raise TrsmError(code, what)


def _torch():
    import torch
    return torch


def colmajor(t):
    """Column-major view or copy of a 2-D tensor (1-D -> one column)."""
    if t.dim() == 1:
        t = t.unsqueeze(1)
    if t.dim() != 2:
        raise ValueError("expected a matrix")
    rows, cols = t.shape
    if t.stride(0) == 1 and (cols <= 1 or t.stride(1) >= max(rows, 1)):
        return t
    return t.t().contiguous().t()


def _ld(t):
    return max(int(t.stride(1)) if t.shape[1] > 1 else int(t.shape[0]), 1)


def _dev_matrix(t, what):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{what} must be float64")
    return colmajor(t)


def _stream(t):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


class Plan:
    """Handle of ``trsm_plan``: L~ resident on the device."""

    def __init__(self, handle, device):
        self._h = ctypes.c_void_p(handle)
        self.device = device
        lib = load_library()
        n, n0, nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib.trsm_plan_sizes(self._h, ctypes.byref(n), ctypes.byref(n0), ctypes.byref(nb)),
               "trsm_plan_sizes")
        self.n, self.n0, self.nblocks = n.value, n0.value, nb.value
        self.sliced = False  # digit planes of the sliced schedule (trsm_plan_sliced)

    @property
    def handle(self):
        return self._h

    def device_bytes(self):
        """Device bytes held by the plan (L~ and any mixed-precision data)."""
        return int(load_library().trsm_plan_device_bytes(self._h))

    def lt(self):
        """L~ as a torch tensor view (n x n, column-major) of the plan's memory."""
        torch = _torch()
        lib = load_library()
        ld = ctypes.c_int64()
        ptr = lib.trsm_plan_lt(self._h, ctypes.byref(ld))

        class _View:
            __cuda_array_interface__ = {
                "shape": (self.n, self.n), "typestr": "<f8",
                "data": (ptr, False), "version": 3,
                "strides": (8, 8 * ld.value),
            }
        return torch.as_tensor(_View(), device=self.device)

    def destroy(self):
        if self._h is not None and self._h.value:
            load_library().trsm_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def trsm_plan(L, n0):
    """Invert the n0 x n0 diagonal blocks of L into a device-resident plan."""
    L = _dev_matrix(L, "L")
    n = L.shape[0]
    if L.shape[1] != n:
        raise ValueError("L must be square")
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.trsm_plan(ctypes.c_void_p(L.data_ptr()), n, _ld(L), int(n0), _stream(L),
                         ctypes.byref(h)), "trsm_plan")
    return Plan(h.value, L.device)


def trsm_solve(plan, B, X=None):
    """X = L^-1 B with a plan; X may be B (in place).  Asynchronous."""
    torch = _torch()
    B = _dev_matrix(B, "B")
    n, k = B.shape
    if n != plan.n:
        raise ValueError("B has the wrong number of rows")
    if X is None:
        X = torch.empty((k, n), dtype=torch.float64, device=B.device).t()
    else:
        X = _dev_matrix(X, "X")
        if X.shape != B.shape:
            raise ValueError("X must have B's shape")
    _check(load_library().trsm_solve(plan.handle, ctypes.c_void_p(B.data_ptr()), k, _ld(B),
                                     ctypes.c_void_p(X.data_ptr()), _ld(X), _stream(B)),
           "trsm_solve")
    return X


def trsm_solve_noalloc(plan, B, X):
    """trsm_solve without device allocation: the workspace is the library's
    fixed 64 MiB scratch array (for callers that may not allocate while
    solving).  Overlapping calls on one device race; larger problems raise
    TrsmError(TRSM_ENOSCRATCH)."""
    B = _dev_matrix(B, "B")
    X = _dev_matrix(X, "X")
    n, k = B.shape
    if n != plan.n or X.shape != B.shape:
        raise ValueError("B and X must be n x k")
    _check(load_library().trsm_solve_noalloc(plan.handle, ctypes.c_void_p(B.data_ptr()), k, _ld(B),
                                             ctypes.c_void_p(X.data_ptr()), _ld(X), _stream(B)),
           "trsm_solve_noalloc")
    return X


def trsm_plan_mixed(plan, L, inner="tf32"):
    """Adds the mixed-precision data (inner = "bf16", "tf32", "bf16x3" or
    "fp16x3", the split updates) to a plan made from L."""
    L = _dev_matrix(L, "L")
    code = {"bf16": TRSM_INNER_BF16, "tf32": TRSM_INNER_TF32, "bf16x3": TRSM_INNER_BF16X3,
            "fp16x3": TRSM_INNER_FP16X3}[inner]
    _check(load_library().trsm_plan_mixed(plan.handle, ctypes.c_void_p(L.data_ptr()), _ld(L), code,
                                          _stream(L)), "trsm_plan_mixed")
    plan.inner = inner
    return plan


def trsm_solve_mixed(plan, B, X=None, residual="sliced", max_iter=30, tol=1e-14, raise_on_noconv=True,
                     s_fp32=False, s_tc=False, s_tc_planes=3):
    """Iterative refinement around the low-precision solve (s_fp32: the
    diagonal multiplies in FP32; s_tc: on the tensor cores as split-tf32
    products of s_tc_planes planes per factor: 3 FP32-class, 2 about
    2^-21, 1 plain tf32).  Returns (X, iterations, last max|D|/max|X|)."""
    torch = _torch()
    B = _dev_matrix(B, "B")
    n, k = B.shape
    if X is None:
        X = torch.empty((k, n), dtype=torch.float64, device=B.device).t()
    else:
        X = _dev_matrix(X, "X")
    it = ctypes.c_int()
    upd = ctypes.c_double()
    code = {"sliced": TRSM_RESIDUAL_SLICED, "fp64": TRSM_RESIDUAL_FP64, "sliced8": TRSM_RESIDUAL_SLICED8,
            "adaptive": TRSM_RESIDUAL_ADAPTIVE, "progressive": TRSM_RESIDUAL_PROGRESSIVE}[residual]
    if s_fp32:
        code |= TRSM_SOLVE_S_FP32
    if s_tc:
        if s_tc_planes not in (1, 2, 3):
            raise ValueError(f"s_tc_planes must be 1, 2 or 3, not {s_tc_planes}")
        code |= {3: TRSM_SOLVE_S_TC, 2: TRSM_SOLVE_S_TC2, 1: TRSM_SOLVE_S_TC1}[s_tc_planes]
    rc = load_library().trsm_solve_mixed(plan.handle, ctypes.c_void_p(B.data_ptr()), k, _ld(B),
                                         ctypes.c_void_p(X.data_ptr()), _ld(X), code, int(max_iter),
                                         float(tol), ctypes.byref(it), ctypes.byref(upd), _stream(B))
    if rc == TRSM_ENOCONV and not raise_on_noconv:
        return X, it.value, upd.value
    _check(rc, "trsm_solve_mixed")
    return X, it.value, upd.value


SCHEDULES = {"dag": 0, "right-looking": 1, "recursive": 2, "sliced": 3}


def trsm_plan_sliced(plan):
    """Adds the digit planes of the sliced schedule to a plan (synchronous;
    a no-op when they are there)."""
    if getattr(plan, "sliced", False):
        return
    torch = _torch()
    s = ctypes.c_void_p(torch.cuda.current_stream(plan.device).cuda_stream)
    _check(load_library().trsm_plan_sliced(plan.handle, s), "trsm_plan_sliced")
    plan.sliced = True


def trsm_solve_schedule(plan, B, X=None, schedule="dag"):
    """trsm_solve with a chosen schedule: "dag" (default persistent
    kernel), "right-looking" (the paper's B~ loop with look-ahead),
    "recursive" (Rec-TRSM) or "sliced" (both matrix multiplies as
    FP64-class digit-sliced tensor-core products; its plan data is made on
    first use).  Asynchronous."""
    torch = _torch()
    if schedule == "sliced":
        trsm_plan_sliced(plan)
    B = _dev_matrix(B, "B")
    n, k = B.shape
    if X is None:
        X = torch.empty((k, n), dtype=torch.float64, device=B.device).t()
    else:
        X = _dev_matrix(X, "X")
    _check(load_library().trsm_solve_schedule(plan.handle, ctypes.c_void_p(B.data_ptr()), k, _ld(B),
                                              ctypes.c_void_p(X.data_ptr()), _ld(X), SCHEDULES[schedule],
                                              _stream(B)), "trsm_solve_schedule")
    return X


def trsm_solve_workspace_size(plan, k):
    out = ctypes.c_size_t()
    _check(load_library().trsm_solve_workspace_size(plan.handle, int(k), ctypes.byref(out)),
           "trsm_solve_workspace_size")
    return out.value


def trsm_solve_ws(plan, B, X, ws):
    """trsm_solve with a caller-provided workspace tensor (uint8, CUDA)."""
    B = _dev_matrix(B, "B")
    X = _dev_matrix(X, "X")
    n, k = B.shape
    _check(load_library().trsm_solve_ws(plan.handle, ctypes.c_void_p(B.data_ptr()), k, _ld(B),
                                        ctypes.c_void_p(X.data_ptr()), _ld(X),
                                        ctypes.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size(),
                                        _stream(B)), "trsm_solve_ws")
    return X


def trsm_sync_status(plan, device=None):
    torch = _torch()
    s = ctypes.c_void_p(torch.cuda.current_stream(device or plan.device).cuda_stream)
    _check(load_library().trsm_sync_status(plan.handle, s), "trsm_sync_status")


def trtri_blocks(L, n0, out=None):
    """Inverses of the diagonal blocks, returned as (N, n0, n0) with out[b]
    the b-th inverse in matrix orientation (a view of the packed buffer)."""
    torch = _torch()
    L = _dev_matrix(L, "L")
    n = L.shape[0]
    n0 = int(n0)
    nb = (n + n0 - 1) // n0
    if out is None:
        out = torch.empty((nb, n0, n0), dtype=torch.float64, device=L.device)
    elif out.numel() < nb * n0 * n0 or not out.is_contiguous() or out.dtype != torch.float64:
        raise ValueError("out must be a contiguous float64 tensor of N*n0*n0 elements")
    _check(load_library().trtri_blocks(ctypes.c_void_p(L.data_ptr()), n, _ld(L), n0,
                                       ctypes.c_void_p(out.data_ptr()), _stream(L)),
           "trtri_blocks")
    # packed block b is column-major n0 x n0: element (r, c) at [b, c, r]
    return out.view(nb, n0, n0).transpose(1, 2)


def trsm_host(L, B, n0, X=None, stream=0):
    """The whole method on host (numpy) buffers through the C ABI: copies in,
    plans, solves, copies out.  Arrays are float64; any layout is accepted
    (converted to Fortran order), pinned memory is not required."""
    L = np.asfortranarray(L, dtype=np.float64)
    B = np.asfortranarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    n, k = B.shape
    if X is None:
        X = np.empty((n, k), dtype=np.float64, order="F")
    _check(load_library().trsm_host(L.ctypes.data, n, max(1, L.shape[0]), int(n0), B.ctypes.data, k,
                                    max(1, n), X.ctypes.data, max(1, n), ctypes.c_void_p(stream)),
           "trsm_host")
    return X


def trsm_host_ptr(L_ptr, n, ldl, n0, B_ptr, k, ldb, X_ptr, ldx, stream=0):
    """trsm_host on raw host pointers (e.g. pinned torch tensors)."""
    _check(load_library().trsm_host(ctypes.c_void_p(L_ptr), n, ldl, int(n0), ctypes.c_void_p(B_ptr),
                                    k, ldb, ctypes.c_void_p(X_ptr), ldx, ctypes.c_void_p(stream)),
           "trsm_host")


def fp64_peak(iters=4096, device=None):
    """Measured FP64 DFMA throughput of the device, TFLOP/s."""
    torch = _torch()
    out = ctypes.c_double()
    s = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    _check(load_library().trsm_fp64_peak(int(iters), ctypes.byref(out), s), "trsm_fp64_peak")
    return out.value


def fp32_peak(iters=8192, device=None):
    """Measured FP32 FFMA throughput of the device, TFLOP/s."""
    torch = _torch()
    out = ctypes.c_double()
    s = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    _check(load_library().trsm_fp32_peak(int(iters), ctypes.byref(out), s), "trsm_fp32_peak")
    return out.value


def workspace_trim(keep_bytes=0):
    """Returns the library's idle workspace memory on the current device to
    the system, keeping at most `keep_bytes` reserved."""
    _check(load_library().trsm_workspace_trim(int(keep_bytes)), "trsm_workspace_trim")


def workspace_reserved_bytes():
    """Bytes the library's workspace pool holds on the current device."""
    return int(load_library().trsm_workspace_reserved_bytes())


def launch_count(reset=False):
    return int(load_library().trsm_launch_count(1 if reset else 0))


class Batch:
    """Many independent systems solved by one persistent launch
    (trsm_batch_*).  `systems` is a list of dicts with keys L (or plan), B,
    X (CUDA tensors, column-major), n0 (32 or 64, plan-less items) and
    optionally tile_cols (columns per output tile: FP64 1 to 3 or a multiple
    of 4 up to 32, FP32 8, 16 or 32; default: fitted to k)."""

    def __init__(self, systems, dtype="f64", arena=None):
        """arena: optional uint8 CUDA tensor to lay the batch out in (no
        allocation); it must hold workspace_size(systems) bytes."""
        torch = _torch()
        items = self._items(systems, dtype)
        h = ctypes.c_void_p()
        code = TRSM_F64 if dtype == "f64" else TRSM_F32
        if arena is None:
            _check(load_library().trsm_batch_create(items, len(systems), code, ctypes.byref(h)), "trsm_batch_create")
        else:
            _check(load_library().trsm_batch_create_ws(items, len(systems), code, ctypes.c_void_p(arena.data_ptr()),
                                                       arena.numel(), self._s(), ctypes.byref(h)),
                   "trsm_batch_create_ws")
            self._keep.append(arena)
        self._h = h

    @staticmethod
    def workspace_size(systems, dtype="f64"):
        b = Batch.__new__(Batch)
        items = b._items(systems, dtype)
        out = ctypes.c_size_t()
        _check(load_library().trsm_batch_workspace_size(items, len(systems), TRSM_F64 if dtype == "f64" else TRSM_F32,
                                                        ctypes.byref(out)), "trsm_batch_workspace_size")
        return out.value

    def _items(self, systems, dtype):
        torch = _torch()
        items = (BatchItem * len(systems))()
        self._keep = []
        want = torch.float64 if dtype == "f64" else torch.float32
        for i, sy in enumerate(systems):
            B, X = colmajor(sy["B"]), colmajor(sy["X"])
            for t in (B, X):
                if not t.is_cuda or t.dtype != want:
                    raise TypeError("batch tensors must be CUDA tensors of the batch dtype")
            n, k = B.shape
            it = items[i]
            if sy.get("plan") is not None:
                it.plan = sy["plan"].handle.value
                it.L, it.ldl, it.n0 = None, 0, 0
            else:
                L = colmajor(sy["L"])
                if L.dtype != want:
                    raise TypeError("L must have the batch dtype")
                it.L, it.ldl, it.n0 = L.data_ptr(), _ld(L), int(sy.get("n0", 32))
                self._keep.append(L)
            it.B, it.ldb, it.X, it.ldx, it.n, it.k = B.data_ptr(), _ld(B), X.data_ptr(), _ld(X), n, k
            it.tile_cols = int(sy.get("tile_cols", 0))
            self._keep += [B, X]
        return items

    def _s(self):
        torch = _torch()
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def run(self):
        _check(load_library().trsm_batch_run(self._h, self._s()), "trsm_batch_run")

    def capture(self):
        _check(load_library().trsm_batch_capture(self._h, self._s()), "trsm_batch_capture")

    def launch_graph(self):
        _check(load_library().trsm_batch_launch_graph(self._h, self._s()), "trsm_batch_launch_graph")

    def status(self):
        item, row = ctypes.c_int(), ctypes.c_int64()
        rc = load_library().trsm_batch_status(self._h, self._s(), ctypes.byref(item), ctypes.byref(row))
        return rc, item.value, row.value

    def workspace_bytes(self):
        return int(load_library().trsm_batch_workspace_bytes(self._h))

    def destroy(self):
        if self._h is not None and self._h.value:
            load_library().trsm_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
