"""The documented size limits and the degenerate sizes, against the oracle:
the float32 DFT at its largest tube length (n = 1024), tGKB at its largest
slice (l = m = 1024) and at n = 1024 (513 Fourier slices, more CTAs than SMs
in the cooperative launch), RT-tSVD with its largest count of right-hand sides
(p = 64), and every solver on a single Fourier slice (n = 1: no conjugate
pairs, no Parseval doubling)."""
import numpy as np
import pytest

import oracle as O
from paper_2110_02485_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL_X = {torch.float64: 1e-10, torch.float32: 1e-5}


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_02485_gb300 import tprod
    tprod.load()
    return tprod


def dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def blur(N, n, seed, noise=1e-2, l=None, general=0.02):
    """A blurred image with noise (the workloads' law) on an N x N x n operator;
    l > N appends rows of a Gaussian operator."""
    T, c = synth.blur_factors(N, 1.3, 3, 1.5, n=n)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    g = np.random.default_rng(seed)
    P = g.standard_normal(A.shape)
    A = A + general * P / np.linalg.norm(P) * np.linalg.norm(A)
    if l is not None and l > N:
        A = np.concatenate([A, 0.3 * g.standard_normal((n, l - N, N))], axis=1)
    X = synth.lateral(synth.synthetic_image(N, n, 3, 1, g))
    Bt = O.tprod(A, X)
    E = g.standard_normal(Bt.shape)
    E = noise * E / np.linalg.norm(E) * np.linalg.norm(Bt)
    return A, Bt + E, float(np.linalg.norm(E))


def test_fft_at_the_float32_tube_length_limit(tp):
    A = np.random.default_rng(3).standard_normal((1024, 3, 7))
    Ad = dev(A, torch.float32)
    Ah = tp.fft(Ad).cpu().numpy()
    ref = O.fft3(Ad.cpu().double().numpy())[:513]
    assert np.abs(Ah - ref).max() <= 2e-6 * 11 * np.abs(ref).max()
    X = tp.ifft(tp.fft(Ad), 1024).cpu().numpy()
    assert np.abs(X - Ad.cpu().numpy()).max() <= 2e-6 * 11 * np.abs(A).max()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_tgkb_at_the_slice_size_limit(tp, dtype):
    """l = m = 1024 on two Fourier slices."""
    A, B, delta = blur(1024, 2, 5)
    Ad, Bd = dev(A, dtype), dev(B, dtype)
    A64, B64 = (x.cpu().double().numpy() for x in (Ad, Bd))
    ref = O.tgkb_solve(A64, B64, delta, 1.1, 12)
    X, info = tp.tgkb_solve(Ad, Bd, delta, 1.1, 12)
    if ref["margin"] > (1e-9 if dtype == torch.float64 else 1e-4):
        assert info["k"] == ref["k"]
        assert rel(X.cpu().numpy(), ref["X"]) <= TOL_X[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_tgkb_with_more_fourier_slices_than_sms(tp, dtype):
    """n = 1024 (513 half-spectrum slices, the float32 tube-length limit;
    float64 takes n = 512, its limit): the cooperative launch holds more CTAs
    than there are SMs."""
    n = 1024 if dtype == torch.float32 else 512
    A, B, delta = blur(8, n, 6)
    Ad, Bd = dev(A, dtype), dev(B, dtype)
    A64, B64 = (x.cpu().double().numpy() for x in (Ad, Bd))
    ref = O.tgkb_solve(A64, B64, delta, 1.1, 8)
    X, info = tp.tgkb_solve(Ad, Bd, delta, 1.1, 8)
    if ref["margin"] > (1e-9 if dtype == torch.float64 else 1e-4):
        assert info["k"] == ref["k"]
        assert rel(X.cpu().numpy(), ref["X"]) <= TOL_X[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_rtsvd_with_the_largest_count_of_right_hand_sides(tp, dtype):
    """p = 64 lateral slices sharing one factorisation and one k."""
    N, n, p = 16, 8, 64
    T, c = synth.blur_factors(N, 1.3, 3, 1.5, n=n)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    g = np.random.default_rng(7)
    A = A + 0.02 * g.standard_normal(A.shape) / np.sqrt(A.size) * np.linalg.norm(A)
    Xt = np.concatenate([synth.lateral(synth.synthetic_image(N, n, 3, 1, g)) for _ in range(p)], axis=2)
    Bt = O.tprod(A, Xt)
    E = g.standard_normal(Bt.shape)
    E = 1e-2 * E / np.linalg.norm(E) * np.linalg.norm(Bt)
    B, delta = Bt + E, float(np.linalg.norm(E))
    Om = g.standard_normal((n, N, N))
    Ad, Bd, Od = dev(A, dtype), dev(B, dtype), dev(Om, dtype)
    A64, B64, O64 = (x.cpu().double().numpy() for x in (Ad, Bd, Od))
    ref = O.rtsvd_solve(A64, B64, O64, delta, 1.1, 0.01 * np.sqrt(O.fro2(A64)), 3, 4, 1, r_max=N)
    X, info = tp.rtsvd_solve(Ad, Bd, Od, delta, 1.1, 3, 4, 1, r_max=N, eps_rel=0.01)
    assert X.shape == (n, N, p)
    assert info["r"] == ref["r"]
    if ref["margin"] > (1e-9 if dtype == torch.float64 else 1e-4):
        assert info["k"] == ref["k"]
        assert rel(X.cpu().numpy(), ref["X"]) <= TOL_X[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_every_solver_on_a_single_fourier_slice(tp, dtype):
    """n = 1: the tensor is one matrix, the DFT the identity."""
    A, B, delta = blur(20, 1, 8, general=0.1)
    Om = np.random.default_rng(9).standard_normal((1, 20, 20))
    Ad, Bd, Od = dev(A, dtype), dev(B, dtype), dev(Om, dtype)
    A64, B64, O64 = (x.cpu().double().numpy() for x in (Ad, Bd, Od))
    tie = 1e-9 if dtype == torch.float64 else 1e-4
    r1 = O.rtsvd_solve(A64, B64, O64, delta, 1.1, 0.01 * np.sqrt(O.fro2(A64)), 3, 4, 1, r_max=20)
    X1, i1 = tp.rtsvd_solve(Ad, Bd, Od, delta, 1.1, 3, 4, 1, r_max=20, eps_rel=0.01)
    assert i1["r"] == r1["r"]
    if r1["margin"] > tie:
        assert i1["k"] == r1["k"] and rel(X1.cpu().numpy(), r1["X"]) <= TOL_X[dtype]
    r2 = O.tgkb_solve(A64, B64, delta, 1.1, 20)
    X2, i2 = tp.tgkb_solve(Ad, Bd, delta, 1.1, 20)
    if r2["margin"] > tie:
        assert i2["k"] == r2["k"] and rel(X2.cpu().numpy(), r2["X"]) <= TOL_X[dtype]
    r3 = O.tgkt_solve(A64, B64, delta, 1.1, 20, 1e-3, 1e9)
    X3, i3 = tp.tgkt_solve(Ad, Bd, delta, 1.1, 20, 1e-3, 1e9)
    if r3["gkb"]["margin"] > tie:
        assert i3["k"] == r3["k"]
        assert abs(np.log10(i3["mu"]) - np.log10(r3["mu"])) <= 1e-3
        assert rel(X3.cpu().numpy(), r3["X"]) <= 10 * TOL_X[dtype]
    r4 = O.ttsvd_solve(A64, B64, delta, 1.1)
    X4, i4 = tp.ttsvd_solve(Ad, Bd, delta, 1.1)
    if r4["margin"] > tie:
        assert i4["k"] == r4["k"] and rel(X4.cpu().numpy(), r4["X"]) <= TOL_X[dtype]
