"""FP64 oracle, part 1: t-product algebra (Section 2).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only the test suite, the smoke check and the
bench's CPU-baseline leg may import it; the library never does.

Layout: a real tensor with l x m frontal slices and n slices is an array of
shape (n, l, m) (frontal slice k at [k]).  Fourier-domain tensors hold all n
slices (the full spectrum), exactly as fft(., [], 3) produces them.

Everything is float64 / complex128.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------
# Mode-3 DFT (Section 2, below Definition 2.1): fft(A, [], 3) is the
# unnormalised DFT along the tubes; ifft carries the 1/n factor.
# --------------------------------------------------------------------------

def fft3(X: np.ndarray) -> np.ndarray:
    """Unnormalised DFT along mode 3 (axis 0 here)."""
    return np.fft.fft(np.asarray(X, dtype=np.complex128), axis=0)


def ifft3(Xh: np.ndarray) -> np.ndarray:
    """Inverse of fft3 (includes 1/n)."""
    return np.fft.ifft(np.asarray(Xh, dtype=np.complex128), axis=0)


def ifft3_real(Xh: np.ndarray) -> np.ndarray:
    """ifft3 of a conjugate-symmetric spectrum: the real tensor it represents."""
    return ifft3(Xh).real


def dft3_naive(X: np.ndarray) -> np.ndarray:
    """The DFT written as its defining sum: Xh[s] = sum_k X[k] exp(-2 pi i s k / n).

    O(n^2); only for pinning fft3 on small n.
    """
    X = np.asarray(X, dtype=np.complex128)
    n = X.shape[0]
    out = np.zeros_like(X)
    for s in range(n):
        for k in range(n):
            out[s] += X[k] * np.exp(-2j * np.pi * s * k / n)
    return out


def fro2(X: np.ndarray) -> float:
    """||X||_F^2 of a real tensor (Section 1)."""
    X = np.asarray(X, dtype=np.float64)
    return float(np.sum(X * X))


def fro2_hat(Xh: np.ndarray) -> float:
    """||X||_F^2 from its full spectrum (Parseval: (1/n) sum_s ||Xh[s]||_F^2)."""
    n = Xh.shape[0]
    return float(np.sum(np.abs(Xh) ** 2) / n)


# --------------------------------------------------------------------------
# t-product (Definition 2.1) and friends.
# --------------------------------------------------------------------------

def tprod(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A * B via the Fourier domain: facewise products of fft3 slices, then ifft3."""
    Ah, Bh = fft3(A), fft3(B)
    Ch = np.matmul(Ah, Bh)
    C = ifft3(Ch)
    if np.isrealobj(A) and np.isrealobj(B):
        return C.real
    return C


def bcirc(A: np.ndarray) -> np.ndarray:
    """Block-circulant matrix of A: block (t, u) = A[(t - u) mod n]."""
    n, l, m = A.shape
    M = np.zeros((n * l, n * m), dtype=A.dtype)
    for t in range(n):
        for u in range(n):
            M[t * l:(t + 1) * l, u * m:(u + 1) * m] = A[(t - u) % n]
    return M


def unfold(B: np.ndarray) -> np.ndarray:
    n, l, m = B.shape
    return B.reshape(n * l, m)


def fold(M: np.ndarray, n: int) -> np.ndarray:
    return M.reshape(n, M.shape[0] // n, M.shape[1])


def tprod_bcirc(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Definition 2.1 directly: tube (i, j) = sum_k A(i,k,:) circ-conv B(k,j,:),
    written as bcirc(A) @ unfold(B).  No Fourier transform involved."""
    return fold(bcirc(A) @ unfold(B), A.shape[0])


def ttranspose(A: np.ndarray) -> np.ndarray:
    """t-transpose (Section 2): transpose every frontal slice, then reverse
    the order of slices 2..n."""
    n = A.shape[0]
    At = np.empty((n, A.shape[2], A.shape[1]), dtype=A.dtype)
    for k in range(n):
        At[k] = A[(-k) % n].T
    return At


def tidentity(m: int, n: int) -> np.ndarray:
    """Identity tensor: first frontal slice I_m, the rest zero (Section 2)."""
    I = np.zeros((n, m, m))
    I[0] = np.eye(m)
    return I


def e1_tube(n: int) -> np.ndarray:
    """The tube e_1 (1 x 1 x n) with (1,1,1) entry one."""
    e = np.zeros((n, 1, 1))
    e[0, 0, 0] = 1.0
    return e


# --------------------------------------------------------------------------
# Normalize (Algorithm "Normalize").  Per Fourier slice j the coefficient is
# a^(j) = ||V^(j)||_2 and the slice is scaled to unit length.  The paper's
# breakdown branch (a^(j) <= tol) substitutes a random unit vector and sets
# a^(j) = 0; here tol = 0 (only an exactly zero slice breaks down) and the
# substitute is the zero vector.  The t-linear solutions built from the
# output do not depend on which vector fills a broken-down slice, because
# its coefficient is zero.
# --------------------------------------------------------------------------

def normalize_hat(Vh: np.ndarray):
    """Fourier-domain Normalize of a lateral slice given as (n, m) or (n, m, 1).

    Returns (Vh_unit, a) with a (n,) real, a >= 0.
    """
    Vh = np.array(Vh, dtype=np.complex128, copy=True)
    n = Vh.shape[0]
    a = np.zeros(n)
    for j in range(n):
        a[j] = np.linalg.norm(Vh[j])
        if a[j] > 0.0:
            Vh[j] = Vh[j] / a[j]
        else:
            Vh[j] = 0.0
            a[j] = 0.0
    return Vh, a


def normalize(X: np.ndarray):
    """Normalize in the spatial domain: X = V * a with ||V|| = 1.

    X is (n, m, 1) real; returns V (n, m, 1) real and the tube a (n, 1, 1).
    """
    Vh, a = normalize_hat(fft3(X))
    V = ifft3_real(Vh)
    a_t = ifft3_real(a.astype(np.complex128)[:, None, None])
    return V, a_t


def tube_norm(X: np.ndarray) -> float:
    """||X|| := ||X^T * X||_F / ||X||_F (Section 3.2, below Algorithm Normalize)."""
    f = np.sqrt(fro2(X))
    if f == 0.0:
        return 0.0
    return float(np.sqrt(fro2(tprod(ttranspose(X), X))) / f)


# --------------------------------------------------------------------------
# tSVD (Section 2, Algorithm 1): one SVD per Fourier slice.
# --------------------------------------------------------------------------

def tsvd_hat(Ah: np.ndarray):
    """Thin SVD of every Fourier slice: returns Uh (n,l,q), S (n,q), Vh (n,m,q)
    with q = min(l, m) and singular values in descending order per slice.

    For a spectrum of real data the factors are made conjugate symmetric
    (slice n-s is the conjugate of slice s; slices 0 and n/2 are real), so
    that their inverse DFTs are real tensors, as Algorithm 1 needs.
    """
    n = Ah.shape[0]
    U, S, VH = np.linalg.svd(Ah, full_matrices=False)
    V = np.conj(np.swapaxes(VH, 1, 2))
    sym = all(np.allclose(Ah[(n - s) % n], np.conj(Ah[s]), rtol=0, atol=1e-12 * (1 + np.abs(Ah).max()))
              for s in range(n))
    if sym:
        for s in range(n // 2 + 1):
            t = (n - s) % n
            if t == s:  # a real slice: take the real SVD
                u, sv, vh = np.linalg.svd(Ah[s].real, full_matrices=False)
                U[s], S[s], V[s] = u, sv, vh.T
            else:
                U[t], S[t], V[t] = np.conj(U[s]), S[s], np.conj(V[s])
    return U, S, V


def tsvd(A: np.ndarray):
    """Full tSVD A = U * S * V^T returned as real tensors (U: l x q x n,
    S: q x q x n f-diagonal, V: m x q x n), via Algorithm 1 with k = q."""
    Uh, S, Vh = tsvd_hat(fft3(A))
    n, q = S.shape
    Sh = np.zeros((n, q, q), dtype=np.complex128)
    for s in range(n):
        Sh[s] = np.diag(S[s])
    return ifft3_real(Uh), ifft3_real(Sh), ifft3_real(Vh)
