"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Every case feeds both sides the same seeded inputs.  The GPU runs in FP64
(to show it computes the same algorithm: agreement to 1e-10) and in FP32
(the product precision: solutions within 1e-5 relative Frobenius error).  Truncation
indices are integers decided by a floating-point threshold; they must match
exactly unless the oracle's margin puts the decision inside the rounding
band of the GPU precision.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2110_02485_gb300 import synth

pytestmark = pytest.mark.gpu

# relative Frobenius tolerances on X against the FP64 oracle: the stated bound for
# float32 solutions (every case measures below 8e-6), and float64 agreement to
# rounding (measured below 1e-13)
TOL_X = {torch.float64: 1e-10, torch.float32: 1e-5}
# decisions closer than this (relative) to tau*delta may legitimately differ
TIE = {torch.float64: 1e-9, torch.float32: 1e-4}


@pytest.fixture(scope="session")
def tp():
    from paper_2110_02485_gb300 import build, tprod
    build.build()
    tprod.load()
    assert torch.cuda.is_available()
    return tprod


def dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rnd(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


# ----------------------------------------------------------------- DFT ----

@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n,l,m", [(1, 3, 5), (2, 4, 4), (3, 7, 2), (5, 6, 9), (8, 33, 3), (17, 5, 13),
                                   (32, 16, 40), (96, 9, 7), (256, 3, 70), (512, 2, 33)])
def test_fft_matches_oracle(tp, dtype, n, l, m):
    A = rnd((n, l, m), n * 7 + l)
    A_dev = dev(A, dtype)
    Ah = tp.fft(A_dev).cpu().numpy()
    ref = O.fft3(A_dev.cpu().double().numpy())[: n // 2 + 1]
    scale = np.abs(ref).max()
    tol = 1e-13 if dtype == torch.float64 else 2e-6 * (1 + np.log2(n))
    assert Ah.shape == ref.shape
    assert np.abs(Ah - ref).max() <= tol * scale
    X = tp.ifft(tp.fft(A_dev), n).cpu().numpy()
    assert np.abs(X - A_dev.cpu().numpy()).max() <= tol * np.abs(A).max()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_ifft_of_a_spectrum_ignores_imaginary_dc_and_nyquist(tp, dtype):
    n, l, m = 8, 3, 4
    g = np.random.default_rng(1)
    Xh = g.standard_normal((n // 2 + 1, l, m)) + 1j * g.standard_normal((n // 2 + 1, l, m))
    cd = torch.complex64 if dtype == torch.float32 else torch.complex128
    X = tp.ifft(torch.from_numpy(Xh).to("cuda", cd), n).cpu().numpy()
    full = np.concatenate([Xh, np.conj(Xh[1:n // 2][::-1])], axis=0)
    full[0] = full[0].real
    full[n // 2] = full[n // 2].real
    ref = O.ifft3_real(full)
    tol = 1e-13 if dtype == torch.float64 else 2e-6
    assert np.abs(X - ref).max() <= tol * np.abs(ref).max()


# ----------------------------------------------------------- t-product ----

@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n,l,kk,m,trans", [(1, 3, 4, 2, 0), (6, 5, 3, 7, 0), (7, 4, 6, 3, 1), (16, 70, 33, 20, 0),
                                            (9, 130, 17, 3, 1), (32, 64, 64, 64, 0)])
def test_tprod_matches_oracle(tp, dtype, n, l, kk, m, trans):
    A = rnd((n, kk, l) if trans else (n, l, kk), 3 + n)
    B = rnd((n, kk, m), 4 + n)
    C = tp.tprod(dev(A, dtype), dev(B, dtype), transA=bool(trans)).cpu().numpy()
    Ad = dev(A, dtype).cpu().double().numpy()
    Bd = dev(B, dtype).cpu().double().numpy()
    ref = O.tprod(O.ttranspose(Ad) if trans else Ad, Bd)
    tol = 1e-12 if dtype == torch.float64 else 5e-6 * np.sqrt(kk)
    assert rel(C, ref) <= tol


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n,l,kk,m,trans", [(7, 4, 6, 3, 2), (5, 9, 4, 6, 3), (16, 70, 33, 20, 2), (1, 2, 3, 4, 3)])
def test_tprod_transposed_b_matches_oracle(tp, dtype, n, l, kk, m, trans):
    """op(B) = B^T (trans bit 1), with or without op(A) = A^T: the adjoint products."""
    A = rnd((n, kk, l) if trans & 1 else (n, l, kk), 5 + n)
    B = rnd((n, m, kk) if trans & 2 else (n, kk, m), 6 + n)
    C = tp.tprod(dev(A, dtype), dev(B, dtype), transA=bool(trans & 1), transB=bool(trans & 2)).cpu().numpy()
    Ad = dev(A, dtype).cpu().double().numpy()
    Bd = dev(B, dtype).cpu().double().numpy()
    ref = O.tprod(O.ttranspose(Ad) if trans & 1 else Ad, O.ttranspose(Bd) if trans & 2 else Bd)
    tol = 1e-12 if dtype == torch.float64 else 5e-6 * np.sqrt(kk)
    assert rel(C, ref) <= tol


def test_tprod_autograd_gradcheck(tp):
    """The t-product's backward (G * B^T, A^T * G on the GPU) against float64
    central differences of the forward (torch.autograd.gradcheck)."""
    g = torch.Generator(device="cpu").manual_seed(3)
    A = torch.randn(5, 3, 4, generator=g, dtype=torch.float64).cuda().requires_grad_()
    B = torch.randn(5, 4, 2, generator=g, dtype=torch.float64).cuda().requires_grad_()
    assert torch.autograd.gradcheck(tp.tprod_ad, (A, B), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,p", [(12, 8, 1), (16, 9, 3), (20, 16, 2)])
def test_rtsvd_adjoint_matches_oracle(tp, dtype, N, n, p):
    """dL/dB = U_k S_k^{-1} V_k^T * G of the GPU solve's factorisation against
    the oracle's, at the same k."""
    A, B, delta = problem(N, n, seed=30 + p, p=p)
    Om = rnd((n, N, N), 13).astype(np.float32)
    tau, eps_rel = 1.1, 0.01
    ref = O.rtsvd_solve(A.astype(np.float64), B.astype(np.float64), Om.astype(np.float64), delta, tau,
                        eps_rel * np.sqrt(O.fro2(A.astype(np.float64))), 3, 4, 1, r_max=N)
    X, info, fac = tp.rtsvd_solve(dev(A, dtype), dev(B, dtype), dev(Om, dtype), delta, tau, 3, 4, 1, r_max=N,
                                  eps_rel=eps_rel, keep=True)
    if not exact_k_required(ref, dtype):
        pytest.skip("truncation index inside the rounding band")
    assert info["k"] == ref["k"]
    G = rnd((n, N, p), 40 + p)
    dB = tp.rtsvd_adjoint(fac, dev(G, dtype)).cpu().numpy()
    want = O.rtsvd_adjoint(ref, dev(G, dtype).cpu().double().numpy())
    assert dB.shape == (n, N, p)
    assert rel(dB, want) <= (1e-9 if dtype == torch.float64 else 1e-4)
    # repeatable: the factorisation is not overwritten
    dB2 = tp.rtsvd_adjoint(fac, dev(G, dtype)).cpu().numpy()
    assert np.array_equal(dB, dB2)


def test_rtsvd_adjoint_central_differences(tp):
    """Float64 central differences of L(B) = <W, X_k(B)> through the C ABI
    against <dL/dB, E> from the adjoint (k unchanged under the perturbation;
    X_k is linear in B at fixed k, so the difference quotient is exact up to
    rounding)."""
    A, B, delta = problem(16, 9, seed=8, p=2)
    Om = rnd((9, 16, 16), 14)
    dt = torch.float64
    kw = dict(r_max=16, eps_rel=0.01)
    X, info, fac = tp.rtsvd_solve(dev(A, dt), dev(B, dt), dev(Om, dt), delta, 1.1, 3, 4, 1, keep=True, **kw)
    g = np.random.default_rng(9)
    W = g.standard_normal(X.shape)
    dB = tp.rtsvd_adjoint(fac, dev(W, dt)).cpu().numpy()
    h = 1e-6 * np.linalg.norm(B)
    for _ in range(64):
        E = g.standard_normal(B.shape)
        E /= np.linalg.norm(E)
        Xp, ip = tp.rtsvd_solve(dev(A, dt), dev(B + h * E, dt), dev(Om, dt), delta, 1.1, 3, 4, 1, **kw)
        Xm, im = tp.rtsvd_solve(dev(A, dt), dev(B - h * E, dt), dev(Om, dt), delta, 1.1, 3, 4, 1, **kw)
        assert ip["k"] == im["k"] == info["k"]
        fd = (np.sum(W * Xp.cpu().numpy()) - np.sum(W * Xm.cpu().numpy())) / (2 * h)
        assert abs(fd - np.sum(dB * E)) <= 1e-7 * max(abs(fd), np.linalg.norm(dB))


def test_rtsvd_autograd_backward_is_the_adjoint(tp):
    """torch.autograd through RtsvdSolve gives rtsvd_adjoint's dL/dB."""
    A, B, delta = problem(12, 8, seed=4, p=2)
    Om = rnd((8, 12, 12), 15)
    dt = torch.float64
    Bt = dev(B, dt).requires_grad_()
    X = tp.rtsvd_solve_ad(dev(A, dt), Bt, dev(Om, dt), delta, 1.1, 3, block=4, r_max=12, eps_rel=0.01)
    W = dev(np.random.default_rng(5).standard_normal(X.shape), dt)
    (W * X).sum().backward()
    _, _, fac = tp.rtsvd_solve(dev(A, dt), dev(B, dt), dev(Om, dt), delta, 1.1, 3, 4, 1, r_max=12, eps_rel=0.01,
                               keep=True)
    assert torch.allclose(Bt.grad, tp.rtsvd_adjoint(fac, W), rtol=0, atol=1e-12 * float(Bt.grad.abs().max()))


@pytest.mark.parametrize("n,l,kk,m,trans", [(8, 256, 256, 16, 0), (8, 256, 256, 16, 1), (5, 128, 40, 8, 0),
                                            (4, 100, 62, 24, 1), (3, 200, 98, 32, 0), (6, 64, 2, 2, 0),
                                            (3, 1, 2, 2, 1), (4, 300, 130, 14, 1), (2, 150, 66, 6, 0),
                                            (7, 37, 300, 10, 1)])
def test_tprod_tensor_core_shapes(tp, n, l, kk, m, trans):
    """Float32 products with at most 32 columns and even leading dimensions run
    on the tensor cores (3xTF32); ragged row, reduction and column counts
    included.  Their error must stay at the float32 level."""
    A = rnd((n, kk, l) if trans else (n, l, kk), 30 + n)
    B = rnd((n, kk, m), 40 + n)
    C = tp.tprod(dev(A, torch.float32), dev(B, torch.float32), transA=bool(trans)).cpu().numpy()
    Ad = dev(A, torch.float32).cpu().double().numpy()
    Bd = dev(B, torch.float32).cpu().double().numpy()
    ref = O.tprod(O.ttranspose(Ad) if trans else Ad, Bd)
    assert rel(C, ref) <= 5e-6 * np.sqrt(kk)


@pytest.mark.parametrize("n,l,kk,m,trans", [(8, 256, 256, 16, 0), (5, 100, 62, 8, 1), (4, 130, 40, 24, 0)])
def test_tprod_tf32_form(tp, n, l, kk, m, trans):
    """TP_TF32 (one tf32 product on the tensor cores): error at the tf32 level
    (inputs rounded to 10 mantissa bits), inside 2e-3, and well above the
    float32 form's on the same inputs, so the form is really in effect."""
    A = rnd((n, kk, l) if trans else (n, l, kk), 50 + n)
    B = rnd((n, kk, m), 60 + n)
    Ad = dev(A, torch.float32).cpu().double().numpy()
    Bd = dev(B, torch.float32).cpu().double().numpy()
    ref = O.tprod(O.ttranspose(Ad) if trans else Ad, Bd)
    c32 = tp.tprod(dev(A, torch.float32), dev(B, torch.float32), transA=bool(trans)).cpu().numpy()
    ctf = tp.tprod(dev(A, torch.float32), dev(B, torch.float32), transA=bool(trans), tf32=True).cpu().numpy()
    e32, etf = rel(c32, ref), rel(ctf, ref)
    assert etf <= 2e-3
    assert etf > 10 * e32


# --------------------------------------------------------------- solvers ----

def problem(N, n=None, seed=5, noise=1e-2, general=0.02, l=None, p=1):
    """Blurred synthetic images plus noise; p > 1 stacks p images as lateral
    slices of B (delta = ||E||_F over all of them)."""
    n = N if n is None else n
    l = N if l is None else l
    T, c = synth.blur_factors(N, 1.3, 3, 1.5, n=n)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    g = np.random.default_rng(seed)
    P = g.standard_normal(A.shape)
    A = A + general * P / np.linalg.norm(P) * np.linalg.norm(A)
    if l > N:  # tall slices: extra rows
        A = np.concatenate([A, 0.3 * g.standard_normal((n, l - N, N))], axis=1)
    Xt = np.concatenate([synth.lateral(synth.synthetic_image(N, n, 3, 1, g)) for _ in range(p)], axis=2)
    Bt = O.tprod_bcirc(A, Xt) if N <= 24 else None
    if Bt is None:
        Bt = O.tprod(A, Xt)
    E = g.standard_normal(Bt.shape)
    E = noise * E / np.linalg.norm(E) * np.linalg.norm(Bt)
    return A.astype(np.float32), (Bt + E).astype(np.float32), float(np.linalg.norm(E))


def res_tol(res, B, dtype):
    """Residual-norm tolerance: relative part plus the rounding floor of
    forming b - A x in the working precision (u * ||B||)."""
    if dtype == torch.float64:
        return 1e-9 * res + 1e-13 * np.linalg.norm(B)
    return 1e-4 * res + 4e-6 * np.linalg.norm(B)


def exact_k_required(out, dtype):
    return out["margin"] > TIE[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,block,q,p_over,eps_rel", [(12, 8, 1, 0, 3, 0.02), (16, 16, 4, 1, 3, 0.01),
                                                        (20, 17, 3, 2, 4, 0.01), (24, 12, 5, 1, 2, 0.005)])
def test_rtsvd_matches_oracle(tp, dtype, N, n, block, q, p_over, eps_rel):
    A, B, delta = problem(N, n)
    Om = rnd((n, N, N), 11).astype(np.float32)
    tau = 1.1
    ref = O.rtsvd_solve(A.astype(np.float64), B.astype(np.float64), Om.astype(np.float64), delta, tau,
                        eps_rel * np.sqrt(O.fro2(A.astype(np.float64))), p_over, block, q, r_max=N)
    X, info, hist = tp.rtsvd_solve(dev(A, dtype), dev(B, dtype), dev(Om, dtype), delta, tau, p_over, block, q,
                                   r_max=N, eps_rel=eps_rel, res_hist=True)
    X = X.cpu().numpy()
    assert info["r"] == ref["r"]
    if exact_k_required(ref, dtype):
        assert info["k"] == ref["k"]
        assert info["status"] == ref["status"]
        assert rel(X, ref["X"]) <= TOL_X[dtype]
    for k, rk in ref["res"].items():
        assert abs(hist[k] - rk) <= res_tol(rk, B, dtype)
    assert np.isclose(info["norm_a2"], O.fro2(A.astype(np.float64)), rtol=1e-6 if dtype == torch.float32 else 1e-12)


@pytest.mark.parametrize("s", [-12, 12])
def test_rtsvd_float32_scaled_problem(tp, s):
    """A and B scaled by 2^s (delta with them): the solution of A X = B is
    unchanged.  The float32 path at l = m = 32 deflates its second block on the
    binary16 tensor-core split, whose operands the kernel rescales by powers of
    two from their measured magnitudes; the scaled solve must still pick the
    oracle's r and k and match the unscaled oracle solution within 1e-5.  At
    2^-12 unscaled binary16 operands would sit in its subnormal range, at 2^12
    the sketch columns pass its largest value.  (The scale stays inside the
    float32 path's range: the small SVD works with squared inner products of
    the factor, fourth powers of the data's magnitude.)"""
    N, n = 32, 8
    A, B, delta = problem(N, n)
    Om = rnd((n, N, N), 11).astype(np.float32)
    ref = O.rtsvd_solve(A.astype(np.float64), B.astype(np.float64), Om.astype(np.float64), delta, 1.1,
                        0.02 * np.sqrt(O.fro2(A.astype(np.float64))), 3, 16, 1, r_max=N)
    assert exact_k_required(ref, torch.float32)
    f = 2.0 ** s
    X, info = tp.rtsvd_solve(dev(A * np.float32(f), torch.float32), dev(B * np.float32(f), torch.float32),
                             dev(Om, torch.float32), delta * f, 1.1, 3, 16, 1, r_max=N, eps_rel=0.02)
    assert info["status"] == 0
    assert info["r"] == ref["r"] and info["k"] == ref["k"]
    assert rel(X.cpu().numpy(), ref["X"]) <= TOL_X[torch.float32]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,block,p,r_max", [(12, 8, 4, 2, 12), (16, 9, 3, 5, 16), (20, 16, 8, 17, 20),
                                               (24, 6, 16, 64, 24)])
def test_rtsvd_several_lateral_slices_match_oracle(tp, dtype, N, n, block, p, r_max):
    """Problem (I6): p lateral slices share the factorisation and one k chosen
    from the Frobenius residual over all slices."""
    A, B, delta = problem(N, n, seed=7 + p, p=p)
    assert B.shape == (n, N, p)
    Om = rnd((n, N, r_max), 12).astype(np.float32)
    tau, p_over, eps_rel = 1.1, 3, 0.01
    ref = O.rtsvd_solve(A.astype(np.float64), B.astype(np.float64), Om.astype(np.float64), delta, tau,
                        eps_rel * np.sqrt(O.fro2(A.astype(np.float64))), p_over, block, 1, r_max=r_max)
    X, info, hist = tp.rtsvd_solve(dev(A, dtype), dev(B, dtype), dev(Om, dtype), delta, tau, p_over, block, 1,
                                   r_max=r_max, eps_rel=eps_rel, res_hist=True)
    X = X.cpu().numpy()
    assert X.shape == (n, N, p)
    assert info["r"] == ref["r"]
    for k, rk in ref["res"].items():
        assert abs(hist[k] - rk) <= res_tol(rk, B, dtype)
    if exact_k_required(ref, dtype):
        assert info["k"] == ref["k"]
        assert info["status"] == ref["status"]
        assert rel(X, ref["X"]) <= TOL_X[dtype]
        # slice j of the joint solve is the k-term filtered solution of slice j alone
        j = p // 2
        Xj = O.rtsvd_solve(A.astype(np.float64), B[:, :, j:j + 1].astype(np.float64), Om.astype(np.float64),
                           delta, tau, eps_rel * np.sqrt(O.fro2(A.astype(np.float64))), p_over, block, 1,
                           r_max=r_max, k_fixed=ref["k"])["X"]
        assert rel(X[:, :, j:j + 1], Xj) <= TOL_X[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,l,p", [(12, 8, None, 1), (16, 9, None, 1), (20, 16, 28, 1), (24, 6, None, 3),
                                     (40, 8, None, 1), (192, 4, None, 1), (256, 3, None, 2)])
def test_ttsvd_matches_oracle(tp, dtype, N, n, l, p):
    """T-tSVD (Section 4.1) through the RT-tSVD path with the t-identity sketch
    against the oracle's full tSVD: the truncation index, the solution and the
    residual at every s.  N = 192 and 256 take ranks beyond the shared-memory
    small SVD (its working copy in global memory).

    At N >= 160 the leading singular values of each Fourier slice cluster
    (relative gaps 5e-4 to 1e-3 against 1e-2 at N = 40): a cut inside the
    cluster separates singular vectors that float32 rounding mixes, so
    single-index residuals there move by about u sqrt(r) / gap (2e-3 at
    N = 256); those are held to twice that bound, computed from the operator's
    own gaps, while the cuts the discrepancy principle weighs (k - 2 .. k + 2)
    and the solution are held to the usual bounds."""
    A, B, delta = problem(N, n, seed=11 + N, l=l, p=p)
    tau = 1.1
    ref = O.ttsvd_solve(A.astype(np.float64), B.astype(np.float64), delta, tau)
    X, info, hist = tp.ttsvd_solve(dev(A, dtype), dev(B, dtype), delta, tau, res_hist=True)
    X = X.cpu().numpy()
    assert X.shape == (n, N, p)
    assert info["r"] == min(A.shape[1], A.shape[2])
    # the oracle forms the residual as sqrt(||B||^2 - ||U_s^T B||^2), which
    # cancels to about sqrt(u) ||B|| near full rank: compare above that floor
    floor = 1e-6 * np.linalg.norm(B)
    clustered = dtype == torch.float32 and N >= 160
    if clustered:  # twice the first-order bound u sqrt(r) / gap, gap the smallest leading relative gap
        S = np.linalg.svd(O.fft3(A.astype(np.float64)), compute_uv=False)
        gap = float(((S[:, :8] - S[:, 1:9]) / S[:, :1]).min())
        loose = float(np.finfo(np.float32).eps) * np.sqrt(info["r"]) / gap
    for k, rk in ref["res"].items():
        if k >= 1 and rk > floor:
            tol = loose * rk if clustered and abs(k - ref["k"]) > 2 else res_tol(rk, B, dtype)
            assert abs(hist[k] - rk) <= tol, k
    if exact_k_required(ref, dtype):
        assert info["k"] == ref["k"]
        assert info["status"] == ref["status"]
        assert rel(X, ref["X"]) <= TOL_X[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,k_max,l", [(12, 8, 12, None), (16, 17, 16, None), (20, 16, 10, 28), (32, 32, 32, None)])
def test_tgkb_matches_oracle(tp, dtype, N, n, k_max, l):
    A, B, delta = problem(N, n, l=l)
    tau = 1.1
    ref = O.tgkb_solve(A.astype(np.float64), B.astype(np.float64), delta, tau, k_max)
    X, info, hist = tp.tgkb_solve(dev(A, dtype), dev(B, dtype), delta, tau, k_max, res_hist=True)
    X = X.cpu().numpy()
    if exact_k_required(ref, dtype):
        assert info["k"] == ref["k"]
        assert info["status"] == ref["status"]
        assert rel(X, ref["X"]) <= TOL_X[dtype]
    for i, ri in ref["res"].items():
        if i <= info["k"]:
            assert abs(hist[i] - ri) <= res_tol(ri, B, dtype)


def problem_p(N, n, levels, seed=21, general=0.02):
    """Blur operator, len(levels) synthetic images as lateral slices, slice j
    with noise of relative level levels[j]; returns A, B, delta_j."""
    T, c = synth.blur_factors(N, 1.3, 3, 1.5, n=n)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    g = np.random.default_rng(seed)
    P = g.standard_normal(A.shape)
    A = A + general * P / np.linalg.norm(P) * np.linalg.norm(A)
    Xt = np.concatenate([synth.lateral(synth.synthetic_image(N, n, 3, 1, g)) for _ in levels], axis=2)
    Bt = O.tprod(A, Xt)
    B, deltas = Bt.copy(), []
    for j, lev in enumerate(levels):
        E = g.standard_normal(Bt[:, :, j].shape)
        E = lev * E / np.linalg.norm(E) * np.linalg.norm(Bt[:, :, j])
        B[:, :, j] += E
        deltas.append(float(np.linalg.norm(E)))
    return A.astype(np.float32), B.astype(np.float32), deltas


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,p,k_max", [(12, 8, 3, 12), (16, 9, 8, 16), (20, 16, 11, 20), (13, 10, 5, 13),
                                         (32, 32, 9, 32)])
def test_tgkb_p_matches_oracle(tp, dtype, N, n, p, k_max):
    """tGKB_p: every lateral slice with its own delta_j and k_j, against the
    oracle's per-slice tGKB.  Float data with odd m (N = 13) runs the
    one-launch-per-slice form, the rest the batched launch (groups of 8)."""
    levels = [(1e-1, 1e-2, 1e-3, 3e-2, 3e-3)[j % 5] for j in range(p)]
    A, B, deltas = problem_p(N, n, levels, seed=N + p)
    tau = 1.1
    ref = O.tgkb_p_solve(A.astype(np.float64), B.astype(np.float64), deltas, tau, k_max)
    X, infos, hist = tp.tgkb_solve(dev(A, dtype), dev(B, dtype), 0.0, tau, k_max, res_hist=True, deltas=deltas)
    X = X.cpu().numpy()
    assert X.shape == (n, N, p) and len(infos) == p and hist.shape == (p, k_max + 1)
    for j in range(p):
        r, info = ref["per_slice"][j], infos[j]
        assert info["tau_delta"] == pytest.approx(tau * deltas[j], rel=1e-15)
        for i, ri in r["res"].items():
            if i <= info["k"]:
                assert abs(hist[j, i] - ri) <= res_tol(ri, B[:, :, j:j + 1], dtype)
        assert all(hist[j, i] == -1.0 for i in range(info["k"] + 1, k_max + 1))
        if exact_k_required(r, dtype):
            assert info["k"] == r["k"], j
            assert info["status"] == r["status"]
            assert rel(X[:, :, j], r["X"][:, :, 0]) <= TOL_X[dtype]
            assert abs(info["residual"] - r["res"][r["k"]]) <= res_tol(r["res"][r["k"]], B[:, :, j:j + 1], dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,p,k_max,levels", [(12, 8, 3, 12, (1e-2, 1e-2, 1e-2)), (16, 9, 5, 16, (3e-2, 1e-2, 1e-3, 1e-1, 3e-3)),
                                                (20, 16, 4, 20, (1e-1, 1e-2, 3e-3, 1e-3)), (13, 10, 3, 13, (1e-2, 1e-3, 1e-2)),
                                                (24, 12, 6, 5, (1e-2, 1e-3, 1e-3, 1e-4, 1e-1, 1e-2))])
def test_nested_tgkb_p_matches_oracle(tp, dtype, N, n, p, k_max, levels):
    """nested_tGKB_p (Algorithm 6) against the oracle: the k each slice ends
    with, its status, its solution, and the projected residuals it tested.
    The last case caps k (k_max = 5) so that slices end NOT_CONVERGED."""
    A, B, deltas = problem_p(N, n, list(levels), seed=N + 3 * p + (3 if N == 20 else 0))
    eta = 1.1
    ref = O.nested_tgkb_p_solve(A.astype(np.float64), B.astype(np.float64), deltas, eta, k_max)
    X, infos, hist = tp.nested_tgkb_solve(dev(A, dtype), dev(B, dtype), deltas, eta, k_max, res_hist=True)
    X = X.cpu().numpy()
    assert X.shape == (n, N, p) and hist.shape == (p, k_max + 1)
    # exact k only while every decision so far sits outside the rounding band
    for j in range(p):
        tdj = eta * deltas[j]
        if min(abs(r - tdj) / tdj for jj in range(j + 1) for r in ref["res"][jj].values()) <= TIE[dtype]:
            break
        assert infos[j]["k"] == ref["k"][j], j
        assert infos[j]["status"] == ref["status"][j]
        assert rel(X[:, :, j], ref["X"][:, :, j]) <= TOL_X[dtype]
        for k, rk in ref["res"][j].items():
            assert abs(hist[j, k] - rk) <= res_tol(rk, B[:, :, j:j + 1], dtype)
        untested = [k for k in range(k_max + 1) if k not in ref["res"][j]]
        assert all(hist[j, k] == -1.0 for k in untested)
    if k_max == 5:
        assert O.STATUS_NOT_CONVERGED in ref["status"]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_tgkb_p_common_delta_and_cap(tp, dtype):
    """tGKB_p with one delta for every slice (delta_p not given) and a step cap
    that some slices reach (NOT_CONVERGED) while others stop earlier."""
    A, B, deltas = problem_p(16, 8, [1e-1, 1e-3, 1e-1, 1e-3, 1e-2, 1e-1], seed=3)
    tau, k_max = 1.1, 4
    d = float(np.median(deltas))
    ref = O.tgkb_p_solve(A.astype(np.float64), B.astype(np.float64), [d] * 6, tau, k_max)
    X, infos = tp.tgkb_solve(dev(A, dtype), dev(B, dtype), d, tau, k_max)
    X = X.cpu().numpy()
    assert {r["status"] for r in ref["per_slice"]} == {O.STATUS_OK, O.STATUS_NOT_CONVERGED}
    for j in range(6):
        r = ref["per_slice"][j]
        if exact_k_required(r, dtype):
            assert infos[j]["k"] == r["k"] and infos[j]["status"] == r["status"]
            assert rel(X[:, :, j], r["X"][:, :, 0]) <= TOL_X[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,k", [(12, 8, 5), (16, 9, 8), (20, 16, 12), (32, 10, 24)])
def test_tgkb_triplets_match_oracle(tp, dtype, N, n, k):
    """t-singular triplets from k tGKB steps (Section 4.3) against the oracle:
    the singular values of every Fourier slice and the rank-one terms
    U_i s_i V_i^H (free of the sign of each singular pair)."""
    A, B, _ = problem(N, n, seed=50 + k)
    ref = O.ritz_triplets(A.astype(np.float64), B.astype(np.float64), k)
    U, S, V = tp.tgkb_triplets(dev(A, dtype), dev(B, dtype), k)
    Uh = O.fft3(U.cpu().double().numpy())
    Vh = O.fft3(V.cpu().double().numpy())
    Sh = O.fft3(S.cpu().double().numpy()[:, None, :])[:, 0, :]
    tol = 1e-9 if dtype == torch.float64 else 2e-3
    smax = ref["S"].max()
    for s in range(n // 2 + 1):
        assert np.abs(Sh[s].imag).max() <= tol * smax
        assert np.abs(Sh[s].real - ref["S"][s]).max() <= tol * smax
        for i in range(k):
            if ref["S"][s, i] < 1e-3 * smax:
                continue  # tiny trailing values: vectors only defined to rounding / gap
            gap = min([abs(ref["S"][s, i] - ref["S"][s, j]) for j in range(k) if j != i] + [smax])
            if gap < 1e-2 * smax:
                continue  # near-ties: the pair is not well defined in float32
            got = np.outer(Uh[s][:, i], Vh[s][:, i].conj())
            want = np.outer(ref["Uh"][s][:, i], ref["Vh"][s][:, i].conj())
            assert np.abs(got - want).max() <= 10 * tol * smax / gap, (s, i)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,k_max,lo,hi", [(12, 8, 12, 1e-3, 1e9), (16, 17, 16, 1e-2, 1e8), (32, 32, 32, 1e-1, 1e9)])
def test_tgkt_matches_oracle(tp, dtype, N, n, k_max, lo, hi):
    A, B, delta = problem(N, n)
    tau = 1.1
    ref = O.tgkt_solve(A.astype(np.float64), B.astype(np.float64), delta, tau, k_max, lo, hi)
    X, info = tp.tgkt_solve(dev(A, dtype), dev(B, dtype), delta, tau, k_max, lo, hi)
    X = X.cpu().numpy()
    g = ref["gkb"]
    if exact_k_required(g, dtype):
        assert info["k"] == ref["k"]
        assert info["status"] == ref["status"]
        assert abs(np.log10(info["mu"]) - np.log10(ref["mu"])) <= (1e-9 if dtype == torch.float64 else 1e-3)
        assert rel(X, ref["X"]) <= TOL_X[dtype]
        assert abs(info["residual"] - ref["residual"]) <= (1e-9 if dtype == torch.float64 else 1e-4) * ref["residual"]


# ------------------------------------------------------------ edge cases ----

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_tgkb_cap_reports_not_converged(tp, dtype):
    A, B, delta = problem(16, 8)
    X, info = tp.tgkb_solve(dev(A, dtype), dev(B, dtype), delta * 1e-6, 1.1, 3)
    ref = O.tgkb_solve(A.astype(np.float64), B.astype(np.float64), delta * 1e-6, 1.1, 3)
    assert info["status"] == O.STATUS_NOT_CONVERGED == ref["status"]
    assert info["k"] == 3 == ref["k"]
    assert rel(X.cpu().numpy(), ref["X"]) <= TOL_X[dtype]


@pytest.mark.parametrize("N,r_max", [(144, 144), (160, 150)])
def test_rtsvd_large_rank_matches_oracle(tp, N, r_max):
    """Float32 RT-tSVD whose rank passes 128 (the small SVD's register form
    with twenty entries per lane), against the oracle on a few Fourier slices."""
    A, B, delta = problem(N, 4, seed=N, noise=1e-4, general=0.05)
    Om = rnd((4, N, r_max), 17).astype(np.float32)
    tau, eps_rel = 1.1, 1e-6
    ref = O.rtsvd_solve(A.astype(np.float64), B.astype(np.float64), Om.astype(np.float64), delta, tau,
                        eps_rel * np.sqrt(O.fro2(A.astype(np.float64))), 200, 16, 1, r_max=r_max)
    X, info, hist = tp.rtsvd_solve(dev(A, torch.float32), dev(B, torch.float32), dev(Om, torch.float32), delta, tau,
                                   200, 16, 1, r_max=r_max, eps_rel=eps_rel, res_hist=True)
    assert ref["r"] > 128 and info["r"] == ref["r"]
    for k, rk in ref["res"].items():
        assert abs(hist[k] - rk) <= res_tol(rk, B, torch.float32) * 10, k
    if exact_k_required(ref, torch.float32):
        assert info["k"] == ref["k"]
        assert rel(X.cpu().numpy(), ref["X"]) <= TOL_X[torch.float32]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_rtsvd_rmax_cap_reports_not_converged(tp, dtype):
    A, B, delta = problem(16, 8)
    Om = rnd((8, 16, 6), 3).astype(np.float32)
    X, info = tp.rtsvd_solve(dev(A, dtype), dev(B, dtype), dev(Om, dtype), delta, 1.1, 2, 2, 1, r_max=6,
                             eps_rel=1e-6)
    ref = O.rtsvd_solve(A.astype(np.float64), B.astype(np.float64), Om.astype(np.float64), delta, 1.1,
                        1e-6 * np.sqrt(O.fro2(A.astype(np.float64))), 2, 2, 1, r_max=6)
    assert info["r"] == 6 == ref["r"]
    assert info["status"] == O.STATUS_NOT_CONVERGED == ref["status"]
    assert info["k"] == ref["k"]
    assert rel(X.cpu().numpy(), ref["X"]) <= TOL_X[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_zero_fourier_slices_break_down_cleanly(tp, dtype):
    """Constant tubes make every Fourier slice but the first exactly zero (for
    a power-of-two n both FFTs produce exact zeros): Normalize breaks down
    there (zero coefficient) and the solvers must still agree with the oracle."""
    n, N = 8, 10
    A = np.tile(rnd((1, N, N), 21) + 3 * np.eye(N), (n, 1, 1))
    B = np.tile(rnd((1, N, 1), 22), (n, 1, 1))
    ref = O.tgkb_solve(A, B, 1e-3, 1.1, N)
    X, info = tp.tgkb_solve(dev(A, dtype), dev(B, dtype), 1e-3, 1.1, N)
    assert info["k"] == ref["k"]
    assert rel(X.cpu().numpy(), ref["X"]) <= TOL_X[dtype]
    Om = rnd((n, N, N), 23)
    refr = O.rtsvd_solve(A, B, Om, 1e-3, 1.1, 1e-3 * np.sqrt(O.fro2(A)), 2, 2, 1, r_max=N)
    Xr, infor = tp.rtsvd_solve(dev(A, dtype), dev(B, dtype), dev(Om, dtype), 1e-3, 1.1, 2, 2, 1, r_max=N,
                               eps_rel=1e-3)
    assert infor["r"] == refr["r"] and infor["k"] == refr["k"]
    assert rel(Xr.cpu().numpy(), refr["X"]) <= TOL_X[dtype]


def test_invalid_arguments_raise(tp):
    A = torch.zeros((4, 5, 5), device="cuda")
    B = torch.zeros((4, 5, 1), device="cuda")
    with pytest.raises(tp.TprodError):
        tp.tgkb_solve(A, B, 1.0, 1.1, 0)
    with pytest.raises(tp.TprodError):
        tp.rtsvd_solve(A, B, torch.zeros((4, 5, 5), device="cuda"), 1.0, 1.1, 2, block=64, r_max=5, eps_rel=0.1)


def test_captured_graph_replay_matches_plain_calls(tp):
    """A solve recorded as a CUDA graph (tprod.Captured) and replayed gives
    the plain call's results bit for bit, and its kernels are this
    library's (counted at capture)."""
    A, B, delta = problem(16, 8, seed=2)
    Om = rnd((8, 16, 16), 3).astype(np.float32)
    dt = torch.float32
    Ad, Bd, Od = dev(A, dt), dev(B, dt), dev(Om, dt)

    def step():
        X1, i1, _ = tp.rtsvd_solve(Ad, Bd, Od, delta, 1.1, 3, 4, 1, r_max=16, eps_rel=0.01, sync=False)
        X2, i2, _ = tp.tgkb_solve(Ad, Bd, delta, 1.1, 16, sync=False)
        X3, i3 = tp.tgkt_solve(Ad, Bd, delta, 1.1, 16, 1e-2, 1e8, sync=False)
        return (X1, X2, X3), (i1, i2, i3)

    ref, rinfo = step()
    ref = [x.clone() for x in ref]
    rinfo = [tp._info_dict(i) for i in rinfo]
    g = tp.Captured(step)
    assert g.launches > 10
    for _ in range(2):
        Xs, infos = g.replay()
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(Xs, ref))
        assert [tp._info_dict(i) for i in infos] == rinfo



# ------------------------------------- gradients in the tube weights c ----

def separable_problem(N, n, seed, p=1, noise=1e-2):
    """A(:,:,k) = c_k T exactly (float64), p blurred images plus noise."""
    T, c = synth.blur_factors(N, 1.3, 3, 1.5, n=n)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    g = np.random.default_rng(seed)
    Xt = np.concatenate([synth.lateral(synth.synthetic_image(N, n, 3, 1, g)) for _ in range(p)], axis=2)
    Bt = O.tprod_bcirc(A, Xt)
    E = g.standard_normal(Bt.shape)
    E = noise * E / np.linalg.norm(E) * np.linalg.norm(Bt)
    return T, c, A, Bt + E, float(np.linalg.norm(E))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,p", [(16, 9, 1), (20, 16, 2), (24, 12, 1)])
def test_sep_grad_c_rtsvd_matches_oracle(tp, dtype, N, n, p):
    """dL/dc of the RT-tSVD solution (k fixed) for L = <W, X_k>, against the
    oracle's gradient of its own solve on the same inputs."""
    T, c, A, B, delta = separable_problem(N, n, 40 + N, p=p)
    if dtype == torch.float32:
        A, B = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
    Om = rnd((n, N, N), 41).astype(np.float32).astype(np.float64)
    ref = O.rtsvd_solve(A, B, Om, delta, 1.1, 0.01 * np.sqrt(O.fro2(A)), 3, 4, 1, r_max=N)
    X, info = tp.rtsvd_solve(dev(A, dtype), dev(B, dtype), dev(Om, dtype), delta, 1.1, 3, 4, 1, r_max=N,
                             eps_rel=0.01)
    if not exact_k_required(ref, dtype):
        pytest.skip("truncation index inside the rounding band")
    assert info["k"] == ref["k"]
    W = rnd((n, N, p), 42)
    dc = tp.sep_grad_c(X, dev(W, dtype), dev(c, torch.float64)).cpu().numpy()
    want = O.grad_c_separable(ref["X"], W, c)
    assert dc.shape == (n,)
    assert rel(dc, want) <= (1e-8 if dtype == torch.float64 else 5e-3)


def test_sep_grad_c_rtsvd_central_differences(tp):
    """Float64 central differences of L(c) = ||X_k(c) - W||^2 through the GPU
    solve (k and the sketch rank unchanged under the perturbation) against
    the GPU gradient.  The sketch stops at rank 20 < 24 by the eta test."""
    N, n = 24, 10
    T, c, A, B, delta = separable_problem(N, n, 50)
    Om = rnd((n, N, N), 51)
    dt = torch.float64
    kw = dict(r_max=N, eps_rel=0.01)
    X, info = tp.rtsvd_solve(dev(A, dt), dev(B, dt), dev(Om, dt), delta, 1.1, 3, 4, 1, **kw)
    W = rnd((n, N, 1), 52)
    G = 2.0 * (X - dev(W, dt))
    dc = tp.sep_grad_c(X, G, dev(c, dt)).cpu().numpy()
    g = np.random.default_rng(53)
    h = 1e-6 * np.linalg.norm(c)
    loss = lambda Xs: float(np.sum((Xs.cpu().numpy() - W) ** 2))
    for _ in range(64):
        e = g.standard_normal(n)
        e /= np.linalg.norm(e)
        Ap = synth.blur_tensor(T, c + h * e, dtype=np.float64)
        Am = synth.blur_tensor(T, c - h * e, dtype=np.float64)
        Xp, ip = tp.rtsvd_solve(dev(Ap, dt), dev(B, dt), dev(Om, dt), delta, 1.1, 3, 4, 1, **kw)
        Xm, im = tp.rtsvd_solve(dev(Am, dt), dev(B, dt), dev(Om, dt), delta, 1.1, 3, 4, 1, **kw)
        assert ip["k"] == im["k"] == info["k"] and ip["r"] == im["r"] == info["r"] == 20
        fd = (loss(Xp) - loss(Xm)) / (2 * h)
        assert abs(fd - dc @ e) <= 1e-6 * max(abs(fd), np.linalg.norm(dc))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,k_max", [(12, 8, 12), (16, 17, 16)])
def test_tgkt_grad_c_matches_oracle(tp, dtype, N, n, k_max):
    """dL/dc of the Tikhonov-tGKB solution (k and mu fixed), damping term
    included, against the oracle's gradient of its own solve."""
    T, c, A, B, delta = separable_problem(N, n, 60 + N)
    if dtype == torch.float32:
        A, B = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
    ref = O.tgkt_solve(A, B, delta, 1.1, k_max, 1e-3, 1e9)
    X, info, fac = tp.tgkt_solve(dev(A, dtype), dev(B, dtype), delta, 1.1, k_max, 1e-3, 1e9, keep=True)
    if not exact_k_required(ref["gkb"], dtype):
        pytest.skip("truncation index inside the rounding band")
    assert info["k"] == ref["k"] and info["status"] == ref["status"] == O.STATUS_OK
    W = rnd((n, N, 1), 61)
    Wd = dev(W, dtype)
    dc = tp.tgkt_grad_c(fac, Wd, dev(c, torch.float64)).cpu().numpy()
    want = O.grad_c_separable(ref["X"], W, c, lam=1.0 / ref["mu"], rho=O.tikhonov_rho(ref["gkb"], ref["mu"], W))
    assert rel(dc, want) <= (1e-6 if dtype == torch.float64 else 3e-2)
    # repeatable: the solve's workspace is only read
    assert np.array_equal(dc, tp.tgkt_grad_c(fac, Wd, dev(c, torch.float64)).cpu().numpy())


def test_tgkt_grad_c_central_differences(tp):
    """Float64 central differences through the GPU Tikhonov-tGKB solve at a
    fixed mu (a search interval whose upper end still leaves the residual
    above tau*delta, so the solve returns mu = mu_hi) against the GPU
    gradient; k unchanged under the perturbation."""
    N, n = 16, 12
    T, c, A, B, delta = separable_problem(N, n, 70)
    dt = torch.float64
    _, free = tp.tgkt_solve(dev(A, dt), dev(B, dt), delta, 1.1, 16, 1e-3, 1e9)
    mu0 = free["mu"] / 20.0
    args = (delta, 1.1, 16, mu0 / 4.0, mu0)
    X, info, fac = tp.tgkt_solve(dev(A, dt), dev(B, dt), *args, keep=True)
    assert info["status"] == O.STATUS_NOT_CONVERGED and abs(info["mu"] / mu0 - 1.0) <= 1e-12
    W = rnd((n, N, 1), 71)
    dc = tp.tgkt_grad_c(fac, dev(W, dt), dev(c, dt)).cpu().numpy()
    g = np.random.default_rng(72)
    h = 1e-6 * np.linalg.norm(c)
    for _ in range(64):
        e = g.standard_normal(n)
        e /= np.linalg.norm(e)
        Xp, ip = tp.tgkt_solve(dev(synth.blur_tensor(T, c + h * e, dtype=np.float64), dt), dev(B, dt), *args)
        Xm, im = tp.tgkt_solve(dev(synth.blur_tensor(T, c - h * e, dtype=np.float64), dt), dev(B, dt), *args)
        assert ip["k"] == im["k"] == info["k"]
        fd = (float(np.sum(W * Xp.cpu().numpy())) - float(np.sum(W * Xm.cpu().numpy()))) / (2 * h)
        assert abs(fd - dc @ e) <= 1e-6 * max(abs(fd), np.linalg.norm(dc))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_sep_grad_c_tgkb_p_matches_oracle(tp, dtype):
    """dL/dc of the tGKB_p solution (every lateral slice with its own k_j)."""
    N, n, p = 16, 10, 3
    T, c = synth.blur_factors(N, 1.3, 3, 1.5, n=n)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    g = np.random.default_rng(80)
    Xt = np.concatenate([synth.lateral(synth.synthetic_image(N, n, 3, 1, g)) for _ in range(p)], axis=2)
    Bt = O.tprod_bcirc(A, Xt)
    E = g.standard_normal(Bt.shape)
    E = 1e-2 * E / np.linalg.norm(E) * np.linalg.norm(Bt)
    deltas = [float(np.linalg.norm(E[:, :, j])) for j in range(p)]
    B = Bt + E
    if dtype == torch.float32:
        A, B = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
    ref = O.tgkb_p_solve(A, B, deltas, 1.1, 12)
    X, infos = tp.tgkb_solve(dev(A, dtype), dev(B, dtype), 0.0, 1.1, 12, deltas=deltas)
    if not all(exact_k_required(o, dtype) for o in ref["per_slice"]):
        pytest.skip("a truncation index inside the rounding band")
    assert [i["k"] for i in infos] == ref["k"]
    W = rnd((n, N, p), 81)
    dc = tp.sep_grad_c(X, dev(W, dtype), dev(c, torch.float64)).cpu().numpy()
    assert rel(dc, O.grad_c_separable(ref["X"], W, c)) <= (1e-8 if dtype == torch.float64 else 5e-3)


@pytest.mark.parametrize("n", [1, 2, 3, 64])
def test_sep_grad_c_ttsvd_tube_lengths(tp, n):
    """dL/dc of the T-tSVD solution for short tubes (one slice; the Nyquist
    slice present or absent) and a longer one, float64."""
    N = 12
    T, c, A, B, delta = separable_problem(N, n, 90 + n)
    ref = O.ttsvd_solve(A, B, delta, 1.1)
    X, info = tp.ttsvd_solve(dev(A, torch.float64), dev(B, torch.float64), delta, 1.1)
    if not exact_k_required(ref, torch.float64):
        pytest.skip("truncation index inside the rounding band")
    assert info["k"] == ref["k"]
    W = rnd((n, N, 1), 91)
    dc = tp.sep_grad_c(X, dev(W, torch.float64), dev(c, torch.float64)).cpu().numpy()
    assert rel(dc, O.grad_c_separable(ref["X"], W, c)) <= 1e-8


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_sep_operator_is_the_blur_tensor(tp, dtype):
    """A(:,:,k) = c_k T with the product in float64 and one rounding: the
    generator's tensor for the T the device holds."""
    T, c = synth.blur_factors(20, 1.3, 3, 1.5, n=9)
    Td = dev(T, dtype)
    A = tp.sep_operator(Td, dev(c, torch.float64)).cpu().numpy()
    assert np.array_equal(A, synth.blur_tensor(Td.cpu().double().numpy(), c, dtype=A.dtype))


def test_sep_rtsvd_autograd_gradcheck(tp):
    """torch.autograd.gradcheck of the RT-tSVD solve in B and c together
    (float64; k = 6 and r = 8 < 10 stay fixed under the perturbations)."""
    T, c, A, B, delta = separable_problem(10, 6, 101)
    Om = dev(rnd((6, 10, 10), 102), torch.float64)
    Td = dev(T, torch.float64)
    Bd = dev(B, torch.float64).requires_grad_()
    cd = dev(c, torch.float64).requires_grad_()
    f = lambda Bx, cx: tp.rtsvd_solve_sep_ad(cx, Td, Bx, Om, delta, 1.1, 3, block=4, q_power=1, r_max=10,
                                             eps_rel=0.01)
    assert torch.autograd.gradcheck(f, (Bd, cd), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_sep_tgkt_autograd_gradcheck(tp):
    """gradcheck of the Tikhonov-tGKB solve in B and c together at a fixed mu
    (the search interval ends below the discrepancy root, so mu = mu_hi under
    every perturbation; k = the discrepancy index stays fixed too)."""
    T, c, A, B, delta = separable_problem(10, 6, 101)
    Td = dev(T, torch.float64)
    Bd = dev(B, torch.float64)
    _, free = tp.tgkt_solve(dev(A, torch.float64), Bd, delta, 1.1, 10, 1e-3, 1e9)
    mu0 = free["mu"] / 20.0
    cd = dev(c, torch.float64).requires_grad_()
    Bg = Bd.clone().requires_grad_()
    f = lambda Bx, cx: tp.tgkt_solve_sep_ad(cx, Td, Bx, delta, 1.1, 10, mu0 / 4.0, mu0)
    assert torch.autograd.gradcheck(f, (Bg, cd), eps=1e-6, atol=1e-7, rtol=1e-5)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,l", [(12, 8, None), (16, 9, None), (20, 16, 28), (32, 32, None)])
def test_tgkt_adjoint_matches_oracle(tp, dtype, N, n, l):
    """dL/dB of the Tikhonov-tGKB solution (Section 5) at the k and mu of the
    GPU solve against the oracle's reverse sweep through Algorithm 4 at the
    same k and mu; repeatable (the solve's workspace is only read)."""
    A, B, delta = problem(N, n, seed=70 + N, l=l)
    Ad, Bd = dev(A, dtype), dev(B, dtype)
    A64, B64 = (x.cpu().double().numpy() for x in (Ad, Bd))
    X, info, fac = tp.tgkt_solve(Ad, Bd, delta, 1.1, min(12, N), 1e-3, 1e9, keep=True)
    k, mu = info["k"], info["mu"]
    ref = O.tgkt_solve(A64, B64, delta, 1.1, min(12, N), 1e-3, 1e9)
    if exact_k_required(ref["gkb"], dtype):
        assert k == ref["k"]
    G = rnd((n, N, 1), 71)
    dB = tp.tgkt_adjoint(fac, dev(G, dtype)).cpu().numpy()
    want, Xo = O.tgkt_adjoint(A64, B64, k, mu, dev(G, dtype).cpu().double().numpy())
    assert dB.shape == (n, A.shape[1], 1)
    assert rel(X.cpu().numpy(), Xo) <= (1e-10 if dtype == torch.float64 else 1e-5)
    assert rel(dB, want) <= (1e-9 if dtype == torch.float64 else 1e-5)
    assert np.array_equal(dB, tp.tgkt_adjoint(fac, dev(G, dtype)).cpu().numpy())


def test_tgkt_adjoint_central_differences_64_directions(tp):
    """The GPU dL/dB (float64) of L = ||X - X_true||_F^2 against FP64 central
    differences (h = 1e-6 relative) of the oracle's Tikhonov-tGKB map at the
    solve's fixed k and mu, on 64 seeded directions."""
    A, B, delta = problem(12, 8, seed=77)
    g = np.random.default_rng(78)
    Xt = g.standard_normal((8, 12, 1))
    X, info, fac = tp.tgkt_solve(dev(A, torch.float64), dev(B, torch.float64), delta, 1.1, 12, 1e-3, 1e9,
                                 keep=True)
    k, mu = info["k"], info["mu"]
    dB = tp.tgkt_adjoint(fac, dev(2.0 * (X.cpu().numpy() - Xt), torch.float64)).cpu().numpy()
    loss = lambda Bv: float(np.sum((O.tgkt_fixed(A, Bv, k, mu) - Xt) ** 2))
    h = 1e-6
    for _ in range(64):
        D = g.standard_normal(B.shape)
        D *= np.linalg.norm(B) / np.linalg.norm(D)
        fd = (loss(B + h * D) - loss(B - h * D)) / (2 * h)
        assert abs(fd - np.sum(dB * D)) <= 1e-7 * np.linalg.norm(dB) * np.linalg.norm(D)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,l", [(12, 8, None), (20, 16, 28), (32, 32, None)])
def test_tgkb_adjoint_matches_oracle(tp, dtype, N, n, l):
    """dL/dB of the tGKB solution (Algorithm 4, Eq. (solgkb)) at the k of the
    GPU solve against the oracle's reverse sweep with no damping (mu = inf)."""
    A, B, delta = problem(N, n, seed=90 + N, l=l)
    Ad, Bd = dev(A, dtype), dev(B, dtype)
    A64, B64 = (x.cpu().double().numpy() for x in (Ad, Bd))
    X, info, fac = tp.tgkb_solve(Ad, Bd, delta, 1.1, min(12, N), keep=True)
    G = rnd((n, N, 1), 91)
    dB = tp.tgkb_adjoint(fac, dev(G, dtype)).cpu().numpy()
    want, Xo = O.tgkt_adjoint(A64, B64, info["k"], np.inf, dev(G, dtype).cpu().double().numpy())
    assert rel(X.cpu().numpy(), Xo) <= (1e-10 if dtype == torch.float64 else 1e-5)
    assert rel(dB, want) <= (1e-9 if dtype == torch.float64 else 1e-5)


def test_tgkb_adjoint_central_differences_64_directions(tp):
    """The GPU dL/dB (float64) of L = <W, X> for the tGKB solution against
    FP64 central differences of the oracle's tGKB at the solve's k, on 64
    seeded directions."""
    A, B, delta = problem(16, 9, seed=93)
    g = np.random.default_rng(94)
    X, info, fac = tp.tgkb_solve(dev(A, torch.float64), dev(B, torch.float64), delta, 1.1, 12, keep=True)
    k = info["k"]
    W = g.standard_normal(X.shape)
    dB = tp.tgkb_adjoint(fac, dev(W, torch.float64)).cpu().numpy()
    loss = lambda Bv: float(np.sum(W * O.tgkb_solve(A, Bv, 0.0, 1.0, k, k_fixed=k)["X"]))
    h = 1e-6
    for _ in range(64):
        D = g.standard_normal(B.shape)
        D *= np.linalg.norm(B) / np.linalg.norm(D)
        fd = (loss(B + h * D) - loss(B - h * D)) / (2 * h)
        assert abs(fd - np.sum(dB * D)) <= 1e-7 * np.linalg.norm(dB) * np.linalg.norm(D)


def test_krylov_autograd_gradcheck_in_B(tp):
    """gradcheck of TgkbSolve (k fixed by the discrepancy principle under the
    perturbations) and TgktSolve (mu = mu_hi: the interval ends below the
    discrepancy root) in B, float64, for a general (non-separable) A."""
    A, B, delta = problem(10, 6, seed=95)
    Ad = dev(A, torch.float64)
    Bg = dev(B, torch.float64).requires_grad_()
    assert torch.autograd.gradcheck(lambda Bx: tp.tgkb_solve_ad(Ad, Bx, delta, 1.1, 10), (Bg,), eps=1e-6,
                                    atol=1e-7, rtol=1e-5)
    _, free = tp.tgkt_solve(Ad, Bg.detach(), delta, 1.1, 10, 1e-3, 1e9)
    mu0 = free["mu"] / 20.0
    assert torch.autograd.gradcheck(lambda Bx: tp.tgkt_solve_ad(Ad, Bx, delta, 1.1, 10, mu0 / 4.0, mu0), (Bg,),
                                    eps=1e-6, atol=1e-7, rtol=1e-5)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_tgkt_adjoint_after_the_hat_solve(tp, dtype):
    """The adjoint of a solve given A-hat (tgkb_tikhonov_solve_hat) reads that
    half spectrum and equals the adjoint of the plain solve."""
    A, B, delta = problem(16, 9, seed=79)
    Ad, Bd = dev(A, dtype), dev(B, dtype)
    G = dev(rnd((9, 16, 1), 80), dtype)
    _, i1, f1 = tp.tgkt_solve(Ad, Bd, delta, 1.1, 12, 1e-3, 1e9, keep=True)
    _, i2, f2 = tp.tgkt_solve(None, Bd, delta, 1.1, 12, 1e-3, 1e9, keep=True, Ahat=tp.fft(Ad), n=9)
    assert i1["k"] == i2["k"]
    d1, d2 = tp.tgkt_adjoint(f1, G).cpu().numpy(), tp.tgkt_adjoint(f2, G).cpu().numpy()
    assert rel(d2, d1) <= (1e-12 if dtype == torch.float64 else 1e-5)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N,n,p", [(12, 8, 1), (16, 9, 2)])
def test_ttsvd_adjoint_matches_oracle(tp, dtype, N, n, p):
    """dL/dB = U_s S_s^{-1} V_s^T * G of the GPU T-tSVD solve against the
    oracle's, at the same s; repeatable (the factorisation is only read)."""
    A, B, delta = problem(N, n, seed=50 + p, p=p)
    ref = O.ttsvd_solve(A.astype(np.float64), B.astype(np.float64), delta, 1.1)
    X, info, fac = tp.ttsvd_solve(dev(A, dtype), dev(B, dtype), delta, 1.1, keep=True)
    if not exact_k_required(ref, dtype):
        pytest.skip("truncation index inside the rounding band")
    assert info["k"] == ref["k"]
    G = rnd((n, N, p), 60 + p)
    dB = tp.ttsvd_adjoint(fac, dev(G, dtype)).cpu().numpy()
    want = O.ttsvd_adjoint(A.astype(np.float64), ref, dev(G, dtype).cpu().double().numpy())
    assert dB.shape == (n, N, p)
    assert rel(dB, want) <= (1e-9 if dtype == torch.float64 else 1e-4)
    assert np.array_equal(dB, tp.ttsvd_adjoint(fac, dev(G, dtype)).cpu().numpy())


# ------------------------------------------------ precomputed A-hat ----

@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_hat_entry_points_match_the_plain_solves_and_the_oracle(tp, dtype):
    """rtsvd_truncated_solve_hat, tgkb_solve_hat and tgkb_tikhonov_solve_hat
    with A-hat from tprod_fft: the plain calls' truncation indices and the
    oracle's solutions (||A||^2 for Algorithm 3 comes from A-hat by Parseval)."""
    A, B, delta = problem(20, 16, seed=21)
    n = A.shape[0]
    Om = rnd((n, 20, 20), 23).astype(np.float32)
    Ad, Bd, Omd = dev(A, dtype), dev(B, dtype), dev(Om, dtype)
    Ah = tp.fft(Ad)
    A64, B64 = (x.astype(np.float64) for x in (A, B))
    eps_rel = 0.02
    ref = O.rtsvd_solve(A64, B64, Om.astype(np.float64), delta, 1.1, eps_rel * np.sqrt(O.fro2(A64)), 3, 4, 1, r_max=20)
    X0, i0 = tp.rtsvd_solve(Ad, Bd, Omd, delta, 1.1, 3, 4, 1, r_max=20, eps_rel=eps_rel)
    X1, i1 = tp.rtsvd_solve(None, Bd, Omd, delta, 1.1, 3, 4, 1, r_max=20, eps_rel=eps_rel, Ahat=Ah, n=n)
    assert (i1["r"], i1["k"], i1["status"]) == (i0["r"], i0["k"], i0["status"]) == (ref["r"], ref["k"], ref["status"])
    assert np.isclose(i1["norm_a2"], O.fro2(A64), rtol=1e-6 if dtype == torch.float32 else 1e-12)
    assert rel(X1.cpu().numpy(), ref["X"]) <= TOL_X[dtype]
    ref = O.tgkb_solve(A64, B64, delta, 1.1, 16)
    X1, i1 = tp.tgkb_solve(None, Bd, delta, 1.1, 16, Ahat=Ah, n=n)
    assert (i1["k"], i1["status"]) == (ref["k"], ref["status"])
    assert rel(X1.cpu().numpy(), ref["X"]) <= TOL_X[dtype]
    ref = O.tgkt_solve(A64, B64, delta, 1.1, 16, 1e-2, 1e8)
    X1, i1 = tp.tgkt_solve(None, Bd, delta, 1.1, 16, 1e-2, 1e8, Ahat=Ah, n=n)
    assert i1["k"] == ref["k"]
    assert rel(X1.cpu().numpy(), ref["X"]) <= TOL_X[dtype]


def test_hat_entry_points_refuse_a_missing_or_mismatched_spectrum(tp):
    A, B, delta = problem(8, 6, seed=2)
    Bd = dev(B, torch.float32)
    Ah = tp.fft(dev(A, torch.float32))
    with pytest.raises(ValueError):
        tp.tgkb_solve(None, Bd, delta, 1.1, 4, Ahat=Ah, n=8)   # 8 // 2 + 1 != 4 slices
    with pytest.raises(ValueError):
        tp.tgkb_solve(None, Bd, delta, 1.1, 4)                 # neither A nor A-hat


# ------------------------------------------------------ BF16 sketch form ----

def test_rtsvd_bf16_form_matches_oracle_within_its_bound(tp):
    """The TP_BF16 form (sketch and power products on bfloat16 copies of A-hat,
    float32 accumulation, float32 re-projection) on the oracle-sized workload
    (config n32): the oracle's sketch rank and truncation index, and the
    solution within the reduced-precision bound 3e-3 (measured 4.9e-5 by a
    bfloat16 emulation of the sketch in float64; on small blur problems whose
    sketch stops just past k + p the bfloat16 error reaches 3e-3 to 1.5e-2, so
    the bound is a property of the workload, not of the products)."""
    P = synth.blur_problem("n32")
    cfg = P["cfg"]
    A64, B64, Om64 = (P[k].astype(np.float64) for k in ("A", "B", "Omega"))
    ref = O.rtsvd_solve(A64, B64, Om64, P["delta"], cfg.tau, cfg.eps_rel * np.sqrt(O.fro2(A64)), cfg.p_over,
                        cfg.block, cfg.q_power, cfg.r_max)
    f = torch.float32
    A, B, Om = dev(P["A"], f), dev(P["B"], f), dev(P["Omega"], f)
    X, info = tp.rtsvd_solve(A, B, Om, P["delta"], cfg.tau, cfg.p_over, cfg.block, cfg.q_power, cfg.r_max,
                             eps_rel=cfg.eps_rel, bf16=True)
    assert info["r"] == ref["r"] and info["k"] == ref["k"]
    assert rel(X.cpu().numpy(), ref["X"]) <= 3e-3
    Xh, ih = tp.rtsvd_solve(None, B, Om, P["delta"], cfg.tau, cfg.p_over, cfg.block, cfg.q_power, cfg.r_max,
                            eps_rel=cfg.eps_rel, bf16=True, Ahat=tp.fft(A), n=cfg.N)
    assert ih["k"] == info["k"] and rel(Xh.cpu().numpy(), ref["X"]) <= 3e-3


def test_rtsvd_bf16_form_refuses_shapes_its_products_do_not_take(tp):
    A, B, delta = problem(18, 8, seed=2)     # 18 complex entries a row: not a multiple of 4
    Om = rnd((8, 18, 18), 3).astype(np.float32)
    f = torch.float32
    with pytest.raises(tp.TprodError):
        tp.rtsvd_solve(dev(A, f), dev(B, f), dev(Om, f), delta, 1.1, 3, 4, 1, r_max=18, eps_rel=0.02, bf16=True)
