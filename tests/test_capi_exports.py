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


def test_product_path_has_no_cpu_fallback():
    """The binding refuses CPU tensors instead of computing on the host."""
    import torch
    from paper_2110_02485_gb300 import tprod
    with pytest.raises(TypeError):
        tprod.fft(torch.zeros(4, 3, 3))


def test_rtsvd_lateral_slice_limits(lib):
    """Workspace sizing (host only) accepts 1 <= p <= 64 lateral slices of B,
    grows with p, and refuses an r_max whose small SVD working set
    (r_max^2 + r_max p complex entries) would not fit in shared memory."""
    from paper_2110_02485_gb300 import build, tprod
    L = tprod.load(build.build())
    P = tprod.RtsvdParams(1.0, 1.1, 0.1, 0.0, 2, 1, 16, 64, None)
    sizes = [L.rtsvd_workspace_bytes(256, 256, 256, p, ctypes.byref(P), tprod.TP_FP32) for p in (1, 2, 17, 64)]
    assert all(s > 0 for s in sizes) and sizes == sorted(sizes) and sizes[0] < sizes[-1]
    for p in (0, 65, -1):
        assert L.rtsvd_workspace_bytes(256, 256, 256, p, ctypes.byref(P), tprod.TP_FP32) == 0
    # FP32 at r_max = 160: 160^2 + 160 p complex64 entries fit for p = 1, not for p = 64
    P.r_max = 160
    assert L.rtsvd_workspace_bytes(256, 256, 256, 1, ctypes.byref(P), tprod.TP_FP32) > 0
    assert L.rtsvd_workspace_bytes(256, 256, 256, 64, ctypes.byref(P), tprod.TP_FP32) == 0
