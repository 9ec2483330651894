"""Pins for the oracle's gradients with respect to the tube weights c of a
separable operator A(:,:,k) = c_k T: float64 central differences of the
oracle's own forward solves (k, the sketch rank and mu held fixed) in seeded
directions (64 of them, as for the gradients in B)."""
import numpy as np
import pytest

import oracle as O
from paper_2110_02485_gb300 import synth


def separable(N, n, seed, noise=1e-2):
    T, c = synth.blur_factors(N, 1.3, 3, 1.5, n=n)
    g = np.random.default_rng(seed)
    Xt = synth.lateral(synth.synthetic_image(N, n, 3, 1, g))
    A = synth.blur_tensor(T, c, dtype=np.float64)
    Bt = O.tprod_bcirc(A, Xt)
    E = g.standard_normal(Bt.shape)
    E = noise * E / np.linalg.norm(E) * np.linalg.norm(Bt)
    return T, c, Bt + E, float(np.linalg.norm(E)), Xt


def fd_check(forward, c, grad, seed, count=64, rtol=1e-6):
    """Central differences of the scalar forward(c) against <grad, e>."""
    g = np.random.default_rng(seed)
    h = 1e-6 * np.linalg.norm(c)
    for _ in range(count):
        e = g.standard_normal(c.shape)
        e /= np.linalg.norm(e)
        fd = (forward(c + h * e) - forward(c - h * e)) / (2 * h)
        assert abs(fd - grad @ e) <= rtol * max(abs(fd), np.linalg.norm(grad))


def test_grad_c_rtsvd_fixed_k_central_differences():
    N, n = 12, 8
    T, c, B, delta, Xt = separable(N, n, 3)
    Om = np.random.default_rng(4).standard_normal((n, N, N))
    A = synth.blur_tensor(T, c, dtype=np.float64)
    ref = O.rtsvd_solve(A, B, Om, delta, 1.1, 0.01 * np.sqrt(O.fro2(A)), 3, 4, 1, r_max=N)
    k, r = ref["k"], ref["r"]
    assert 1 <= k < r
    G = 2.0 * (ref["X"] - Xt)                       # L = ||X_k - X_true||_F^2

    def loss(cc):
        out = O.rtsvd_solve(synth.blur_tensor(T, cc, dtype=np.float64), B, Om, delta, 1.1, 0.0, 3, 4, 1,
                            r_max=r, k_fixed=k)
        return float(np.sum((out["X"] - Xt) ** 2))

    assert np.isclose(loss(c), np.sum((ref["X"] - Xt) ** 2), rtol=1e-12)
    fd_check(loss, c, O.grad_c_separable(ref["X"], G, c), 5)


def test_grad_c_tgkb_and_ttsvd_fixed_k_central_differences():
    N, n = 10, 6
    T, c, B, delta, Xt = separable(N, n, 7)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    W = np.random.default_rng(8).standard_normal((n, N, 1))   # L = <W, X_k>
    g = O.tgkb_solve(A, B, delta, 1.1, 8)
    t = O.ttsvd_solve(A, B, delta, 1.1)
    for out, fwd in ((g, lambda cc: O.tgkb_solve(synth.blur_tensor(T, cc, dtype=np.float64), B, delta, 1.1, 8,
                                                 k_fixed=g["k"])["X"]),
                     (t, lambda cc: O.ttsvd_solve(synth.blur_tensor(T, cc, dtype=np.float64), B, delta, 1.1,
                                                  k_fixed=t["k"])["X"])):
        assert out["k"] >= 1
        fd_check(lambda cc: float(np.sum(W * fwd(cc))), c, O.grad_c_separable(out["X"], W, c), 9)


def test_grad_c_tikhonov_fixed_mu_central_differences():
    N, n = 10, 6
    T, c, B, delta, Xt = separable(N, n, 11)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    tk = O.tgkt_solve(A, B, delta, 1.1, 8, 1e-3, 1e5)
    k, mu = tk["k"], tk["mu"]
    W = np.random.default_rng(12).standard_normal((n, N, 1))

    def fwd(cc):
        g = O.tgkb_solve(synth.blur_tensor(T, cc, dtype=np.float64), B, delta, 1.1, 8, k_fixed=k)
        return O.tikhonov_fixed_mu(g, mu)[0]

    assert np.allclose(fwd(c), tk["X"], rtol=0, atol=1e-12 * np.abs(tk["X"]).max())
    rho = O.tikhonov_rho(tk["gkb"], mu, W)
    grad = O.grad_c_separable(tk["X"], W, c, lam=1.0 / mu, rho=rho)
    fd_check(lambda cc: float(np.sum(W * fwd(cc))), c, grad, 13)
    # the damping term matters: without it the gradient is off
    bare = O.grad_c_separable(tk["X"], W, c)
    assert np.linalg.norm(bare - grad) > 1e-3 * np.linalg.norm(grad)


def test_tikhonov_rho_is_the_mu_derivative():
    """rho_s against central differences of tikhonov_fixed_mu in lam = 1/mu."""
    N, n = 10, 6
    T, c, B, delta, Xt = separable(N, n, 15)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    g = O.tgkb_solve(A, B, delta, 1.1, 7, k_fixed=7)
    G = np.random.default_rng(16).standard_normal((n, N, 1))
    mu = 50.0
    lam, h = 1.0 / mu, 1e-6 / mu
    Xp = O.tikhonov_fixed_mu(g, 1.0 / (lam + h))[0]
    Xm = O.tikhonov_fixed_mu(g, 1.0 / (lam - h))[0]
    dXh = (O.fft3(Xp) - O.fft3(Xm))[:, :, 0] / (2 * h)
    want = np.einsum("si,si->s", np.conj(O.fft3(G)[:, :, 0]), dXh)
    got = O.tikhonov_rho(g, mu, G)
    assert np.allclose(got, want, rtol=1e-6, atol=1e-6 * np.abs(want).max())


def test_grad_c_fails_for_a_non_separable_operator():
    """The identity needs every slice to be a multiple of one T: with a dense
    perturbation added to A the formula no longer gives the derivative in c
    (of A(c) = c_k T + P)."""
    N, n = 10, 6
    T, c, B, delta, Xt = separable(N, n, 17)
    P = 0.3 * np.random.default_rng(18).standard_normal((n, N, N)) * np.abs(T).max()
    A = synth.blur_tensor(T, c, dtype=np.float64) + P
    t = O.ttsvd_solve(A, B, delta, 1.1)
    W = np.random.default_rng(19).standard_normal((n, N, 1))
    grad = O.grad_c_separable(t["X"], W, c)
    e = np.random.default_rng(20).standard_normal(n)
    h = 1e-6
    fwd = lambda cc: float(np.sum(W * O.ttsvd_solve(synth.blur_tensor(T, cc, dtype=np.float64) + P, B, delta, 1.1,
                                                    k_fixed=t["k"])["X"]))
    fd = (fwd(c + h * e) - fwd(c - h * e)) / (2 * h)
    assert abs(fd - grad @ e) > 1e-3 * abs(fd)


def test_grad_c_tgkb_p_central_differences():
    """tGKB_p: every lateral slice has its own Krylov space and k_j, and each
    is a separable solve, so the same formula holds for all p at once."""
    N, n, p = 10, 6, 3
    T, c = synth.blur_factors(N, 1.3, 3, 1.5, n=n)
    g = np.random.default_rng(21)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    Xt = np.concatenate([synth.lateral(synth.synthetic_image(N, n, 3, 1, g)) for _ in range(p)], axis=2)
    Bt = O.tprod_bcirc(A, Xt)
    E = g.standard_normal(Bt.shape)
    E = 1e-2 * E / np.linalg.norm(E) * np.linalg.norm(Bt)
    deltas = [float(np.linalg.norm(E[:, :, j])) for j in range(p)]
    B = Bt + E
    out = O.tgkb_p_solve(A, B, deltas, 1.1, 8)
    W = g.standard_normal((n, N, p))

    def loss(cc):
        o = O.tgkb_p_solve(synth.blur_tensor(T, cc, dtype=np.float64), B, deltas, 1.1, 8)
        assert o["k"] == out["k"]
        return float(np.sum(W * o["X"]))

    fd_check(loss, c, O.grad_c_separable(out["X"], W, c), 22)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_grad_c_short_tubes(n):
    """n = 1 (one slice, dL/dc = -gamma_0 / c), n = 2 and 3 (the Nyquist slice
    and its absence) against central differences of the T-tSVD."""
    N = 8
    T, c, B, delta, Xt = separable(N, n, 23 + n)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    t = O.ttsvd_solve(A, B, delta, 1.1)
    W = np.random.default_rng(24).standard_normal((n, N, 1))
    fwd = lambda cc: float(np.sum(W * O.ttsvd_solve(synth.blur_tensor(T, cc, dtype=np.float64), B, delta, 1.1,
                                                    k_fixed=t["k"])["X"]))
    grad = O.grad_c_separable(t["X"], W, c)
    fd_check(fwd, c, grad, 25)
    if n == 1:
        assert np.isclose(grad[0], -np.sum(W * t["X"]) / c[0], rtol=1e-12)
