"""Pins for the oracle's t-product algebra (Section 2, Algorithm Normalize,
Algorithm 1, Theorem 2.1) against definitions, brute force and closed forms."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2110_02485_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rnd(shape, seed, cplx=False):
    g = np.random.default_rng(seed)
    x = g.standard_normal(shape)
    if cplx:
        x = x + 1j * g.standard_normal(shape)
    return x


# ---------------------------------------------------------------- DFT ----

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 17])
def test_fft3_is_the_defining_sum(n):
    X = rnd((n, 3, 2), n, cplx=True)
    assert np.allclose(O.fft3(X), O.dft3_naive(X), rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [1, 4, 7, 16])
def test_dft_roundtrip_parseval_and_symmetry(n):
    X = rnd((n, 4, 3), 10 + n)
    Xh = O.fft3(X)
    assert np.allclose(O.ifft3_real(Xh), X, atol=1e-13)
    assert np.isclose(O.fro2(X), O.fro2_hat(Xh), rtol=1e-13)
    for s in range(n):           # real data -> conjugate-symmetric spectrum
        assert np.allclose(Xh[(n - s) % n], np.conj(Xh[s]), atol=1e-12)


def test_dft_sign_convention_on_a_shifted_impulse():
    # x_k = delta_{k,1}  ->  xh_s = exp(-2 pi i s / n)   (MATLAB fft convention)
    n = 6
    X = np.zeros((n, 1, 1))
    X[1] = 1.0
    expect = np.exp(-2j * np.pi * np.arange(n) / n)
    assert np.allclose(O.fft3(X)[:, 0, 0], expect, atol=1e-14)


# ----------------------------------------------------------- t-product ----

def test_tprod_golden_hand_example():
    """Definition 2.1 worked by hand on 2x2x2 * 2x1x2 tensors."""
    with open(os.path.join(GOLDEN, "tprod_2x2x2.json")) as f:
        g = json.load(f)
    A = np.array(g["A"], dtype=float)
    B = np.array(g["B"], dtype=float)
    C = np.array(g["C"], dtype=float)
    assert np.allclose(O.tprod(A, B), C, atol=1e-13)
    assert np.allclose(O.tprod_bcirc(A, B), C, atol=1e-13)
    t = g["tube_case"]
    x = np.array(t["x"], dtype=float)[:, None, None]
    y = np.array(t["y"], dtype=float)[:, None, None]
    assert np.allclose(O.tprod(x, y)[:, 0, 0], t["xy"], atol=1e-12)
    assert np.allclose(O.tprod_bcirc(x, y)[:, 0, 0], t["xy"], atol=1e-12)


@pytest.mark.parametrize("n,l,p,m", [(1, 2, 3, 2), (5, 3, 4, 2), (6, 4, 4, 4), (7, 2, 5, 3)])
def test_fourier_tprod_equals_block_circulant(n, l, p, m):
    A = rnd((n, l, p), 1)
    B = rnd((n, p, m), 2)
    assert np.allclose(O.tprod(A, B), O.tprod_bcirc(A, B), atol=1e-12)


def test_tprod_associative():
    A, B, C = rnd((5, 3, 4), 3), rnd((5, 4, 2), 4), rnd((5, 2, 3), 5)
    assert np.allclose(O.tprod(O.tprod(A, B), C), O.tprod(A, O.tprod(B, C)), atol=1e-12)


def test_transpose_identity_and_definition():
    A, B = rnd((6, 3, 4), 6), rnd((6, 4, 2), 7)
    lhs = O.ttranspose(O.tprod(A, B))
    rhs = O.tprod(O.ttranspose(B), O.ttranspose(A))
    assert np.allclose(lhs, rhs, atol=1e-12)
    # the t-transpose is the tensor whose block-circulant is bcirc(A)^T
    assert np.allclose(O.bcirc(O.ttranspose(A)), O.bcirc(A).T)
    # in the Fourier domain it is the conjugate transpose of every slice
    Ah, Ath = O.fft3(A), O.fft3(O.ttranspose(A))
    assert np.allclose(Ath, np.conj(np.swapaxes(Ah, 1, 2)), atol=1e-12)


def test_tproduct_adjoint_is_the_t_transpose():
    """<G, A * B> = <A^T * G, B> = <G * B^T, A>: the t-transpose is the adjoint
    of the t-product in both arguments (the gradient rules of the t-product)."""
    g = np.random.default_rng(12)
    A, B, G = g.standard_normal((5, 3, 4)), g.standard_normal((5, 4, 2)), g.standard_normal((5, 3, 2))
    lhs = np.sum(G * O.tprod_bcirc(A, B))
    assert np.isclose(lhs, np.sum(O.tprod_bcirc(O.ttranspose(A), G) * B), rtol=1e-12)
    assert np.isclose(lhs, np.sum(O.tprod_bcirc(G, O.ttranspose(B)) * A), rtol=1e-12)


def test_identity_tensor():
    A = rnd((5, 3, 4), 8)
    assert np.allclose(O.tprod(O.tidentity(3, 5), A), A, atol=1e-13)
    assert np.allclose(O.tprod(A, O.tidentity(4, 5)), A, atol=1e-13)


# ------------------------------------------------------------- Normalize ----

def test_normalize_contract():
    X = rnd((7, 5, 1), 9)
    V, a = O.normalize(X)
    assert np.allclose(O.tprod(V, a), X, atol=1e-12)          # X = V * a
    assert np.isclose(O.tube_norm(V), 1.0, atol=1e-12)        # ||V|| = 1
    # Eq. (tfrobX): ||X||_F = sqrt((X^T * X)^(1))
    g = O.tprod(O.ttranspose(X), X)
    assert np.isclose(np.sqrt(g[0, 0, 0]), np.sqrt(O.fro2(X)), rtol=1e-12)


def test_normalize_breakdown_slice():
    # constant tubes: only the DC Fourier slice is non-zero
    n = 6
    X = np.tile(rnd((1, 4, 1), 11), (n, 1, 1))
    Vh, a = O.normalize_hat(O.fft3(X))
    assert np.all(a[1:] == 0.0) and a[0] > 0
    assert np.all(Vh[1:] == 0.0)
    V, at = O.normalize(X)
    assert np.allclose(O.tprod(V, at), X, atol=1e-12)


# ------------------------------------------------------------------ tSVD ----

def test_tsvd_orthogonality_and_reconstruction():
    A = rnd((6, 4, 4), 12)
    U, S, V = O.tsvd(A)
    I = O.tidentity(4, 6)
    assert np.allclose(O.tprod(O.ttranspose(U), U), I, atol=1e-12)
    assert np.allclose(O.tprod(O.ttranspose(V), V), I, atol=1e-12)
    # reconstruction through the block-circulant product (no FFT)
    R = O.tprod_bcirc(O.tprod_bcirc(U, S), O.ttranspose(V))
    assert np.allclose(R, A, atol=1e-12)


def test_theorem_2_1_error_with_squared_singular_values():
    n, l, m, k = 5, 6, 4, 2
    A = rnd((n, l, m), 13)
    Uh, S, Vh = O.tsvd_hat(O.fft3(A))
    Akh = Uh[:, :, :k] @ (S[:, :k, None] * np.conj(np.swapaxes(Vh[:, :, :k], 1, 2)))
    err2 = O.fro2(A - O.ifft3_real(Akh))
    assert np.isclose(err2, np.sum(S[:, k:] ** 2) / n, rtol=1e-12)
    # and the unsquared sum printed in the theorem does not match
    assert not np.isclose(err2, np.sum(S[:, k:]) / n, rtol=1e-3)


def test_tsvd_closed_form_for_the_blur_operator():
    """A(:,:,k) = c_k T  =>  sigma_j^(s) = |c_hat_s| * |lambda_j(T)| (T symmetric)."""
    T, c = synth.blur_factors(12, 1.5, 4, 2.0)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    _, S, _ = O.tsvd_hat(O.fft3(A))
    lam = np.sort(np.abs(np.linalg.eigvalsh(T)))[::-1]
    chat = O.dft3_naive(c[:, None, None])[:, 0, 0]
    expect = np.abs(chat)[:, None] * lam[None, :]
    assert np.allclose(S, expect, rtol=1e-10, atol=1e-13)


def test_generator_forward_blur_is_the_tproduct():
    T, c = synth.blur_factors(8, 1.5, 3, 2.0, n=6)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    img = rnd((8, 6), 14)
    B = synth.forward_blur(T, c, img)
    assert np.allclose(synth.lateral(B), O.tprod_bcirc(A, synth.lateral(img)), atol=1e-12)
