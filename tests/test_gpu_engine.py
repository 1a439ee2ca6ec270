"""The tcgen05 tile engine (TMA -> shared memory -> tcgen05.mma -> TMEM ->
epilogue) against a plain FP64 product of the same rounded inputs."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(lib, tf32, M, N, K, seed):
    import torch
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, size=(M, K)).astype(np.float32)
    B = rng.uniform(-1, 1, size=(N, K)).astype(np.float32)
    if tf32:
        At = torch.from_numpy(A).cuda()
        Bt = torch.from_numpy(B).cuda()
        # the tensor core reads the top 19 bits of each fp32 (tf32)
        Ar = (A.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
        Br = (B.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
    else:
        At = torch.from_numpy(A).cuda().to(torch.bfloat16)
        Bt = torch.from_numpy(B).cuda().to(torch.bfloat16)
        Ar = At.float().cpu().numpy()
        Br = Bt.float().cpu().numpy()
    C = torch.full((N, M), float("nan"), dtype=torch.float32, device="cuda")  # column-major M x N
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.trsm_tc_gemm_selftest(int(tf32), ctypes.c_void_p(At.data_ptr()), ctypes.c_void_p(Bt.data_ptr()),
                                   ctypes.c_void_p(C.data_ptr()), M, N, K, ctypes.c_void_p(err.data_ptr()), s)
    assert rc == 0
    torch.cuda.synchronize()
    assert err.item() == 0
    got = C.cpu().numpy().T
    want = Ar.astype(np.float64) @ Br.astype(np.float64).T
    scale = np.abs(Ar).astype(np.float64) @ np.abs(Br).astype(np.float64).T
    return got, want, scale


@pytest.mark.parametrize("tf32", [0, 1])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (128, 128, 32), (300, 200, 520), (1024, 512, 1024),
                                   (64, 16, 8), (129, 257, 200), (129, 300, 1032),
                                   # several tiles per persistent CTA (two TMEM buffers alternating),
                                   # ragged edges, short and long K
                                   (5000, 3000, 1040), (4200, 2100, 96)])
def test_engine_gemm(cuda_lib, tf32, M, N, K):
    if K % (4 if tf32 else 8):
        pytest.skip("K not a multiple of the TMA row granule")
    got, want, scale = _run(cuda_lib, tf32, M, N, K, seed=M + N + K)
    # inputs are exact in the MMA; only FP32 accumulation order differs
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - want) / (scale + 1e-30)) < 2e-6


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 200, 520), (1024, 512, 1024), (129, 257, 200),
                                   (256, 64, 256), (129, 300, 1032), (5000, 3000, 1040), (4200, 2100, 96)])
def test_engine_split_gemm(cuda_lib, M, N, K, fmt):
    """Split operands (hi + lo planes of bf16 or fp16): C = Ah Bh^T + Ah Bl^T + Al Bh^T."""
    import torch
    rng = np.random.default_rng(M * N + K)
    A = rng.uniform(-1, 1, size=(M, K))
    B = rng.uniform(-1, 1, size=(N, K))
    dt = torch.bfloat16 if fmt == "bf16" else torch.float16

    def split(X):
        hi = torch.from_numpy(X).to(dt)
        lo = torch.from_numpy(X - hi.double().numpy()).to(dt)
        return hi, lo

    Ah, Al = split(A)
    Bh, Bl = split(B)
    At = torch.stack([Ah, Al]).contiguous().cuda()  # [2][M][K]
    Bt = torch.stack([Bh, Bl]).contiguous().cuda()
    C = torch.full((N, M), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = cuda_lib.trsm_tc_gemm_selftest(2 if fmt == "bf16" else 3, ctypes.c_void_p(At.data_ptr()),
                                        ctypes.c_void_p(Bt.data_ptr()),
                                        ctypes.c_void_p(C.data_ptr()), M, N, K, ctypes.c_void_p(err.data_ptr()), s)
    assert rc == 0
    torch.cuda.synchronize()
    assert err.item() == 0
    got = C.cpu().numpy().T.astype(np.float64)
    ah, al, bh, bl = (t.double().numpy() for t in (Ah, Al, Bh, Bl))
    three = ah @ bh.T + ah @ bl.T + al @ bh.T
    scale = np.abs(A) @ np.abs(B).T
    # the three products exactly, up to FP32 accumulation
    assert np.max(np.abs(got - three) / scale) < 2e-6
    # against the unsplit FP64 product: the dropped lo*lo term and the
    # representation hi + lo (about 2^-16 each), far below bf16's 2^-8
    rel = np.max(np.abs(got - A @ B.T) / scale)
    assert rel < (2.0 ** -14 if fmt == "bf16" else 2.0 ** -19), rel
