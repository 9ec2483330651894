"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/tprod.h declares (no GPU needed; nothing is computed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "tprod.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2110_02485_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("tprod_fft", "tprod_ifft", "tprod_gemm", "rtsvd_truncated_solve", "tgkb_solve",
              "tgkb_tikhonov_solve"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2110_02485_gb300 import tprod
    assert sorted(tprod.EXPORTS) == declared_functions()


def test_argument_errors_are_synchronous_and_enqueue_nothing(lib):
    lib.tprod_fft.restype = ctypes.c_int
    lib.tprod_fft.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                              ctypes.c_int, ctypes.c_void_p]
    # null pointers / bad sizes / bad precision are rejected before any CUDA call
    assert lib.tprod_fft(None, 4, 4, 4, None, 0, None) == -1
    assert lib.tprod_fft(ctypes.c_void_p(256), 0, 4, 4, ctypes.c_void_p(256), 0, None) == -1
    assert lib.tprod_fft(ctypes.c_void_p(256), 4, 4, 4, ctypes.c_void_p(256), 7, None) == -1
    lib.tp_status_string.restype = ctypes.c_char_p
    assert lib.tp_status_string(-5).decode().startswith("discrepancy")


def test_noalloc_refuses_sizes_whose_scratch_need_would_wrap(lib):
    """Sizes whose byte count would wrap size_t are argument errors, returned
    before any CUDA call (on a host without a GPU a CUDA call would give -2)."""
    f = lib.tprod_gemm_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 6 + [ctypes.c_void_p]
    p = ctypes.c_void_p(256)
    big = 1 << 30
    for prec in (0, 1):
        assert f(p, p, p, big, big, big, 1, 0, prec, None) == -1
        assert f(p, p, p, big, big, 1, 1, 1, prec, None) == -1
        assert f(p, p, p, 1, big, big, 1, 0, prec, None) == -1
    assert f(p, p, p, 65535 * 128 + 1, 1, 1, 1, 0, 0, None) == -1


def test_product_path_has_no_cpu_fallback():
    """The binding refuses CPU tensors instead of computing on the host."""
    import torch
    from paper_2110_02485_gb300 import tprod
    with pytest.raises(TypeError):
        tprod.fft(torch.zeros(4, 3, 3))
    X = torch.zeros(4, 3, 1)
    c = torch.ones(4, dtype=torch.float64)
    with pytest.raises(TypeError):
        tprod.sep_grad_c(X, X, c)
    with pytest.raises(TypeError):
        tprod.sep_operator(torch.zeros(3, 3), c)
    with pytest.raises(TypeError):
        tprod.rtsvd_solve(torch.zeros(4, 3, 3), X, torch.zeros(4, 3, 3), 1.0, 1.1, 1, r_max=3, eps_rel=0.1)


def test_rtsvd_lateral_slice_limits(lib):
    """Workspace sizing (host only) accepts 1 <= p <= 64 lateral slices of B,
    grows with p, and refuses r_max beyond 256 or one whose right-hand sides
    (r_max p complex entries, kept in shared memory by the small SVD also when
    R's working copy moves to global memory) would not fit."""
    from paper_2110_02485_gb300 import build, tprod
    L = tprod.load(build.build())
    P = tprod.RtsvdParams(1.0, 1.1, 0.1, 0.0, 2, 1, 16, 64, None)
    sizes = [L.rtsvd_workspace_bytes(256, 256, 256, p, ctypes.byref(P), tprod.TP_FP32) for p in (1, 2, 17, 64)]
    assert all(s > 0 for s in sizes) and sizes == sorted(sizes) and sizes[0] < sizes[-1]
    for p in (0, 65, -1):
        assert L.rtsvd_workspace_bytes(256, 256, 256, p, ctypes.byref(P), tprod.TP_FP32) == 0
    # FP32 at r_max = 160 and 256: R in shared memory for p = 1, in global memory for p = 64 (160 x 64 and
    # 256 x 64 complex64 right-hand sides fit); FP64 at r_max = 256, p = 64: 256 x 64 complex128 do not
    for r in (160, 256):
        P.r_max = r
        assert L.rtsvd_workspace_bytes(256, 256, 256, 1, ctypes.byref(P), tprod.TP_FP32) > 0
        assert L.rtsvd_workspace_bytes(256, 256, 256, 64, ctypes.byref(P), tprod.TP_FP32) > 0
    assert L.rtsvd_workspace_bytes(256, 256, 256, 64, ctypes.byref(P), tprod.TP_FP64) == 0
    assert L.rtsvd_workspace_bytes(256, 256, 256, 8, ctypes.byref(P), tprod.TP_FP64) > 0
    P.r_max = 257
    assert L.rtsvd_workspace_bytes(512, 512, 256, 1, ctypes.byref(P), tprod.TP_FP32) == 0


def test_workspace_queries_refuse_out_of_range_requests(lib):
    """The host-only workspace queries of the later entry points: zero (the
    refusal) outside each documented limit, positive inside it."""
    from paper_2110_02485_gb300 import build, tprod
    L = tprod.load(build.build())
    T = tprod.TtsvdParams(1.0, 1.1, None)
    assert L.ttsvd_workspace_bytes(64, 64, 32, 1, ctypes.byref(T), tprod.TP_FP32) > 0
    assert L.ttsvd_workspace_bytes(256, 256, 32, 1, ctypes.byref(T), tprod.TP_FP32) > 0    # R in global memory
    assert L.ttsvd_workspace_bytes(256, 256, 32, 1, ctypes.byref(T), tprod.TP_FP64) > 0
    assert L.ttsvd_workspace_bytes(300, 300, 32, 1, ctypes.byref(T), tprod.TP_FP32) == 0   # min(l, m) > 256
    assert L.tgkb_triplets_workspace_bytes(64, 64, 32, 20, tprod.TP_FP32) > 0
    assert L.tgkb_triplets_workspace_bytes(256, 256, 32, 200, tprod.TP_FP32) == 0           # (k+1)^2 too large
    assert L.tgkb_triplets_workspace_bytes(16, 16, 8, 17, tprod.TP_FP32) == 0               # k > min(l, m)
    G = tprod.TgkbParams(1.0, 1.1, 10, None, None)
    assert L.nested_tgkb_workspace_bytes(64, 64, 32, 5, ctypes.byref(G), tprod.TP_FP32) > 0
    assert L.nested_tgkb_workspace_bytes(64, 64, 32, 0, ctypes.byref(G), tprod.TP_FP32) == 0
    assert L.tgkb_workspace_bytes(64, 64, 32, 1025, ctypes.byref(G), tprod.TP_FP32) == 0    # p > 1024
    d = (ctypes.c_double * 2)(1.0, -1.0)                                                    # a negative bound
    Gd = tprod.TgkbParams(1.0, 1.1, 10, None, ctypes.cast(d, ctypes.c_void_p))
    assert L.tgkb_workspace_bytes(64, 64, 32, 2, ctypes.byref(Gd), tprod.TP_FP32) == 0
    K = tprod.TikParams(G, 1e-2, 1e2, 0.0)
    assert L.tgkb_tikhonov_workspace_bytes(64, 64, 32, 2, ctypes.byref(K), tprod.TP_FP32) == 0  # p = 1 only


def test_tube_weight_gradient_queries_and_argument_checks(lib):
    """Workspace queries of the separable-operator gradients, and their
    argument errors, answered on the host (no GPU needed)."""
    from paper_2110_02485_gb300 import tprod
    L = tprod.load()
    assert L.sep_grad_c_workspace_bytes(256, 256, 1, tprod.TP_FP32) > 0
    assert L.sep_grad_c_workspace_bytes(256, 256, 32, tprod.TP_FP64) > L.sep_grad_c_workspace_bytes(
        256, 256, 32, tprod.TP_FP32)
    assert L.sep_grad_c_workspace_bytes(256, 2048, 1, tprod.TP_FP32) == 0                   # n > 1024
    assert L.sep_grad_c_workspace_bytes(0, 16, 1, tprod.TP_FP32) == 0
    assert L.sep_grad_c_workspace_bytes(16, 16, 1, 9) == 0                                  # bad precision
    G = tprod.TgkbParams(1.0, 1.1, 10, None)
    K = tprod.TikParams(G, 1e-2, 1e2, 0.0)
    assert L.tgkb_tikhonov_grad_c_workspace_bytes(64, 64, 32, ctypes.byref(K), tprod.TP_FP32) > 0
    assert L.tgkb_tikhonov_grad_c_workspace_bytes(64, 64, 2048, ctypes.byref(K), tprod.TP_FP32) == 0
    assert L.tgkb_tikhonov_grad_c_workspace_bytes(8, 8, 32, ctypes.byref(K), tprod.TP_FP32) == 0  # k_max > 8
    # null pointers are rejected before any CUDA call
    p = ctypes.c_void_p(256)
    assert L.sep_grad_c(None, p, p, 16, 16, 1, p, tprod.TP_FP32, p, 1 << 20, None) == -1
    assert L.sep_grad_c(p, p, None, 16, 16, 1, p, tprod.TP_FP32, p, 1 << 20, None) == -1
    assert L.tgkb_tikhonov_grad_c(None, p, 64, 64, 32, ctypes.byref(K), p, 1 << 30, p, tprod.TP_FP32, p, 1 << 20,
                                  None) == -1


def test_autotune_table_host_checks(lib):
    """tp_autotune_set answers on the host: shapes the tensor-core product
    does not take and stage counts outside its range are refused, accepted
    entries appear in the table, and clearing empties it."""
    from paper_2110_02485_gb300 import tprod
    L = tprod.load()
    L.tp_autotune_clear()
    assert L.tp_autotune_set(1, 3, 16, 256, 256, 129, 2) == -1        # op T is not a tensor-core form
    assert L.tp_autotune_set(0, 2, 16, 256, 256, 129, 2) == -1        # passes 2 does not exist
    assert L.tp_autotune_set(0, 3, 33, 256, 256, 129, 2) == -1        # more than 32 columns
    assert L.tp_autotune_set(0, 3, 16, 256, 256, 129, 1) == -1        # one stage is no ring
    assert L.tp_autotune_set(0, 3, 16, 256, 256, 129, 7) == -1        # more stages than any CTA holds
    assert L.tp_autotune_set(3, 0, 16, 256, 256, 129, 2) == -1        # the bfloat16 form takes no A^H
    assert L.tp_autotune_set(0, 3, 16, 256, 256, 129, 3) == 0
    assert L.tp_autotune_set(2, 0, 16, 256, 256, 129, 4) == 0
    table = tprod.autotune_table()
    assert {(e["op"], e["form"], e["stages"]) for e in table} == {("A", "fp32", 3), ("conj(A)", "bf16", 4)}
    tprod.autotune_clear()
    assert tprod.autotune_table() == []
