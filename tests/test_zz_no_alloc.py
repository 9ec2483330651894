"""The no-allocation t-product entry point (tprod_gemm_noalloc).

Callers that cannot allocate device memory (no cudaMalloc, no workspace to
hand over) use this entry point; it computes in a fixed 16 MiB scratch array
inside the library.  The test calls it through the C ABI twice in a row, so
the second call runs on the scratch the first left behind, and checks both
results against tprod_gemm with a caller workspace, within the FP32/FP64
t-product tolerances of the parity tests, and one FP64 result against a
t-product the test forms itself (FFT along the tubes, a product per slice,
inverse FFT).  It also checks the edge of the 16 MiB scratch: the largest
cube that fits is computed correctly and the next size up is refused before
anything is written.

This file sorts last so that a run stopping at the first failure has run every
other test first; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2110_02485_gb300 import build, tprod
    build.build()
    L = tprod.load()
    return tprod, L


def call_noalloc(L, A, B, C, transA, prec):
    n, a1, a2 = A.shape
    _, kk, m = B.shape
    l = a2 if transA else a1
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.tprod_gemm_noalloc(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                ctypes.c_void_p(C.data_ptr()), l, kk, m, n, int(transA), prec, stream)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_noalloc_matches_workspace_entry_point_on_two_calls(lib, dtype):
    tprod, L = lib
    prec = 0 if dtype == torch.float32 else 1
    g = np.random.default_rng(7)
    shapes = [((16, 24, 20), (16, 20, 12), False), ((9, 30, 17), (9, 30, 5), True)]
    for (sa, sb, trans) in shapes:  # two calls in a row on the shared scratch
        A = torch.from_numpy(g.standard_normal(sa)).to("cuda", dtype)
        B = torch.from_numpy(g.standard_normal(sb)).to("cuda", dtype)
        ref = tprod.tprod(A, B, transA=trans)
        C = torch.full_like(ref, float("nan"))
        assert call_noalloc(L, A, B, C, trans, prec) == 0
        torch.cuda.synchronize()
        kk = sb[1]
        tol = 1e-12 if dtype == torch.float64 else 5e-6 * np.sqrt(kk)
        err = float(torch.linalg.norm(C - ref) / torch.linalg.norm(ref))
        assert err <= tol


def test_noalloc_rejects_problems_beyond_the_scratch(lib):
    tprod, L = lib
    # three spectra of 33 x 256 x 256 complex64 need about 52 MB > 16 MiB
    A = torch.zeros((64, 256, 256), device="cuda")
    B = torch.zeros((64, 256, 256), device="cuda")
    C = torch.full((64, 256, 256), 3.0, device="cuda")
    assert call_noalloc(L, A, B, C, False, 0) == tprod.TP_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert bool(torch.all(C == 3.0))


def test_noalloc_matches_an_independent_fp64_tproduct(lib):
    tprod, L = lib
    g = np.random.default_rng(11)
    A64 = torch.from_numpy(g.standard_normal((10, 13, 7)))
    B64 = torch.from_numpy(g.standard_normal((10, 7, 6)))
    # facewise product of the Fourier slices (Section 2), formed here with torch.fft on the host
    ref = torch.fft.ifft(torch.fft.fft(A64, dim=0) @ torch.fft.fft(B64, dim=0), dim=0).real
    A, B = A64.to("cuda"), B64.to("cuda")
    C = torch.full((10, 13, 6), float("nan"), device="cuda", dtype=torch.float64)
    assert call_noalloc(L, A, B, C, False, 1) == 0
    torch.cuda.synchronize()
    assert float(torch.linalg.norm(C.cpu() - ref) / torch.linalg.norm(ref)) <= 1e-12


def test_noalloc_at_the_edge_of_the_scratch(lib):
    """n = 16 (9 spectral slices), FP32, cubes of side L: three spectra of
    align256(9 L^2 8) bytes each.  L = 278 needs 16,694,016 bytes (fits in
    16 MiB = 16,777,216); L = 279 needs 16,813,824 (refused)."""
    tprod, L = lib
    g = np.random.default_rng(5)
    side = 278
    A = torch.from_numpy(g.standard_normal((16, side, side))).to("cuda", torch.float32)
    B = torch.from_numpy(g.standard_normal((16, side, side))).to("cuda", torch.float32)
    ref = tprod.tprod(A, B)
    C = torch.full_like(ref, float("nan"))
    assert call_noalloc(L, A, B, C, False, 0) == 0
    torch.cuda.synchronize()
    err = float(torch.linalg.norm(C - ref) / torch.linalg.norm(ref))
    assert err <= 5e-6 * np.sqrt(side)
    side = 279
    A = torch.zeros((16, side, side), device="cuda")
    C = torch.full((16, side, side), 3.0, device="cuda")
    assert call_noalloc(L, A, A, C, False, 0) == tprod.TP_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert bool(torch.all(C == 3.0))
