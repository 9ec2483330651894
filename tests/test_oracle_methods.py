"""Pins for the oracle's solvers: Algorithm 3 and Theorems 4.1/4.2, the
RT-tSVD and T-tSVD methods with the discrepancy principle (Eq. (disp)),
Algorithm 4 and the tGKB method, the Tikhonov variant and t-Lanczos.

Each pin checks the oracle against something other than itself: the
block-circulant product of Definition 2.1 (no Fourier transform), explicit
Krylov bases, dense per-slice solves, or an independent path of the paper.
"""
import numpy as np
import pytest

import oracle as O
from paper_2110_02485_gb300 import synth


def rnd(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def spatial(Xh):
    return O.ifft3_real(Xh)


def small_blur(N=10, n=8, seed=3, noise=1e-2, general=0.0):
    T, c = synth.blur_factors(N, 1.2, 3, 1.5, n=n)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    g = np.random.default_rng(seed)
    if general:
        P = g.standard_normal(A.shape)
        A = A + general * P / np.linalg.norm(P) * np.linalg.norm(A)
    img = synth.synthetic_image(N, n, 3, 1, g)
    Bt = synth.lateral(synth.forward_blur(T, c, img))
    E = g.standard_normal(Bt.shape)
    E = noise * E / np.linalg.norm(E) * np.linalg.norm(Bt)
    return A, Bt + E, float(np.linalg.norm(E))


# ------------------------------------------------------ R-tSVD (Alg. 3) ----

@pytest.mark.parametrize("form", ["alg3", "block"])
def test_theorem_4_2_eta_is_the_approximation_error(form):
    n, l, m = 6, 9, 7
    A = rnd((n, l, m), 1)
    Om = rnd((n, m, m), 2)
    eps = 0.2 * np.sqrt(O.fro2(A))
    if form == "alg3":
        f = O.rtsvd_alg3(A, Om, eps)
        step = 1
    else:
        f = O.rtsvd_block(A, Om, eps, b=2, q=1, r_max=m)
        step = 2
    assert f["eta"] < eps ** 2
    for i, eta in enumerate(f["etas"]):
        r = min(i * step, f["r"])
        Q = spatial(f["Q"][:, :, :r])
        Bt = spatial(f["Bt"][:, :r, :])
        approx = O.tprod_bcirc(Q, Bt) if r else np.zeros_like(A)
        assert np.isclose(eta, O.fro2(A - approx), rtol=1e-9, atol=1e-10 * O.fro2(A))
    # Q is partially orthogonal: Q^T * Q = I (Section 2)
    Q = spatial(f["Q"])
    assert np.allclose(O.tprod_bcirc(O.ttranspose(Q), Q), O.tidentity(f["r"], n), atol=1e-10)


def test_block_form_with_b1_q0_is_algorithm_3():
    n, l, m = 5, 8, 6
    A = rnd((n, l, m), 4)
    Om = rnd((n, m, m), 5)
    eps = 0.1 * np.sqrt(O.fro2(A))
    a = O.rtsvd_alg3(A, Om, eps)
    b = O.rtsvd_block(A, Om, eps, b=1, q=0, r_max=m)
    assert a["r"] == b["r"]
    assert np.allclose(a["Q"], b["Q"], atol=1e-9)
    assert np.allclose(a["Bt"], b["Bt"], atol=1e-9)
    assert np.allclose(a["etas"], b["etas"], rtol=1e-9)


@pytest.mark.parametrize("q_power,block", [(0, 1), (1, 3), (2, 4)])
def test_full_rank_rtsvd_equals_ttsvd_at_every_k(q_power, block):
    """With r = m and A of full tubal rank the R-tSVD factorisation is exact,
    so the RT-tSVD solution at any fixed k is the T-tSVD solution (Eq. (14))."""
    A, B, delta = small_blur(N=8, n=6, general=0.05)
    n, l, m = A.shape
    Om = rnd((n, m, m), 6)
    for k in [1, 3, 5, m]:
        x1 = O.rtsvd_solve(A, B, Om, delta, 1.1, 0.0, m, block, q_power, r_max=m, k_fixed=k)
        x2 = O.ttsvd_solve(A, B, delta, 1.1, k_fixed=k)
        assert x1["r"] == m
        assert np.allclose(x1["X"], x2["X"], atol=1e-8 * np.abs(x2["X"]).max())


def test_rtsvd_discrepancy_residual_and_bracket():
    A, B, delta = small_blur(N=10, n=8, general=0.02)
    n, l, m = A.shape
    Om = rnd((n, m, m), 7)
    tau = 1.1
    out = O.rtsvd_solve(A, B, Om, delta, tau, 0.02 * np.sqrt(O.fro2(A)), 3, 2, 1, r_max=m)
    assert out["status"] == O.STATUS_OK
    for k, rk in out["res"].items():          # residual is ||B - A*X_k|| with the true A
        Xk = O.rtsvd_solve(A, B, Om, delta, tau, 0.02 * np.sqrt(O.fro2(A)), 3, 2, 1,
                           r_max=m, k_fixed=k)["X"]
        assert np.isclose(rk, np.sqrt(O.fro2(B - O.tprod_bcirc(A, Xk))), rtol=1e-9)
    k = out["k"]
    assert out["k_init"] == max(1, out["r"] - 3)
    assert out["res"][k] <= tau * delta
    assert all(out["res"][j] > tau * delta for j in range(out["k_init"], k))


def test_rtsvd_prefix_is_the_sketch_stopped_by_its_eta_test():
    """A prefix of a factorisation sketched to r_max is what the block sketch
    returns when eta falls below eps^2 right after that many columns: the same
    Q, Bt, r and eta, and the same solve."""
    A, B, delta = small_blur(N=10, n=8, general=0.02)
    n, l, m = A.shape
    Om = rnd((n, m, m), 9)
    full = O.rtsvd_block(A, Om, 0.0, 2, 1, m)
    etas = full["etas"]
    for nb in (2, 3):
        # an eps between eta after nb blocks and eta after nb - 1 stops the sketch at r = 2 nb
        eps = np.sqrt(np.sqrt(etas[nb] * etas[nb - 1]))
        ref = O.rtsvd_block(A, Om, eps, 2, 1, m)
        pre = O.rtsvd_prefix(full, 2 * nb, 2)
        assert ref["r"] == pre["r"] == 2 * nb
        assert np.allclose(ref["Q"], pre["Q"], atol=1e-13) and np.allclose(ref["Bt"], pre["Bt"], atol=1e-13)
        assert np.isclose(ref["eta"], pre["eta"], rtol=1e-12)
        a = O.rtsvd_solve(A, B, Om, delta, 1.1, eps, 1, 2, 1, r_max=m)
        b = O.rtsvd_solve(A, B, Om, delta, 1.1, eps, 1, 2, 1, r_max=m, fac=pre)
        assert a["k"] == b["k"] and a["status"] == b["status"]
        assert np.allclose(a["X"], b["X"], atol=1e-12)


def small_blur_multi(p=3, N=10, n=8, seed=13, noise=1e-2, general=0.02):
    """p lateral slices (different images) blurred by one operator, with noise
    of total relative level `noise` (delta = ||E||_F over all slices)."""
    T, c = synth.blur_factors(N, 1.2, 3, 1.5, n=n)
    A = synth.blur_tensor(T, c, dtype=np.float64)
    g = np.random.default_rng(seed)
    P = g.standard_normal(A.shape)
    A = A + general * P / np.linalg.norm(P) * np.linalg.norm(A)
    Xt = np.concatenate([synth.lateral(synth.synthetic_image(N, n, 3, 1, g)) for _ in range(p)], axis=2)
    Bt = O.tprod_bcirc(A, Xt)
    E = g.standard_normal(Bt.shape)
    E = noise * E / np.linalg.norm(E) * np.linalg.norm(Bt)
    return A, Bt + E, float(np.linalg.norm(E))


def test_rtsvd_several_lateral_slices_share_k_and_match_columnwise():
    """Reading for B with p lateral slices (problem (I6)): one factorisation,
    one truncation index k from ||B - A*X_k||_F <= tau delta with delta the
    norm of all of E.  At any fixed k the solution is the column-wise one
    (X_k = V_k S_k^-1 U_k^T * B is linear in B), and the reported residual is
    the Frobenius norm over all slices, checked through the block-circulant
    product."""
    A, B, delta = small_blur_multi(p=3)
    n, l, m = A.shape
    Om = rnd((n, m, m), 8)
    tau, eps = 1.1, 0.02 * np.sqrt(O.fro2(A))
    out = O.rtsvd_solve(A, B, Om, delta, tau, eps, 3, 2, 1, r_max=m)
    assert out["status"] == O.STATUS_OK
    k = out["k"]
    for c in range(3):
        xc = O.rtsvd_solve(A, B[:, :, c:c + 1], Om, delta, tau, eps, 3, 2, 1, r_max=m, k_fixed=k)["X"]
        assert np.allclose(out["X"][:, :, c:c + 1], xc, atol=1e-10 * np.abs(xc).max())
    for j, rj in out["res"].items():
        Xj = O.rtsvd_solve(A, B, Om, delta, tau, eps, 3, 2, 1, r_max=m, k_fixed=j)["X"]
        assert np.isclose(rj, np.sqrt(O.fro2(B - O.tprod_bcirc(A, Xj))), rtol=1e-9)
    assert out["res"][k] <= tau * delta
    assert all(out["res"][j] > tau * delta for j in range(out["k_init"], k))


def test_rtsvd_duplicated_lateral_slice_gives_the_single_slice_answer():
    """B = [b, b] with delta scaled by sqrt(2) is the single-slice problem twice:
    same k, and both solution slices equal the single-slice solution."""
    A, B, delta = small_blur(N=10, n=8, general=0.02)
    n, l, m = A.shape
    Om = rnd((n, m, m), 9)
    tau, eps = 1.1, 0.02 * np.sqrt(O.fro2(A))
    one = O.rtsvd_solve(A, B, Om, delta, tau, eps, 3, 2, 1, r_max=m)
    two = O.rtsvd_solve(A, np.concatenate([B, B], axis=2), Om, np.sqrt(2.0) * delta, tau, eps, 3, 2, 1, r_max=m)
    assert two["k"] == one["k"] and two["r"] == one["r"]
    for c in range(2):
        assert np.allclose(two["X"][:, :, c:c + 1], one["X"], atol=1e-10 * np.abs(one["X"]).max())


def test_rtsvd_adjoint_satisfies_the_adjoint_identity():
    """At fixed k, B -> X_k is linear; its adjoint must satisfy
    <G, X_k(E)> = <adjoint(G), E> for any E and G (real inner products), the
    forward side computed by the solver itself on E.  Also pinned: the
    adjoint of a p-slice G is the slice-wise adjoint."""
    A, B, delta = small_blur_multi(p=2)
    n, l, m = A.shape
    Om = rnd((n, m, m), 10)
    tau, eps = 1.1, 0.02 * np.sqrt(O.fro2(A))
    out = O.rtsvd_solve(A, B, Om, delta, tau, eps, 3, 2, 1, r_max=m)
    k = out["k"]
    g = np.random.default_rng(77)
    for _ in range(3):
        E = g.standard_normal((n, l, 2))
        G = g.standard_normal((n, m, 2))
        XE = O.rtsvd_solve(A, E, Om, delta, tau, eps, 3, 2, 1, r_max=m, k_fixed=k)["X"]
        adj = O.rtsvd_adjoint(out, G)
        assert adj.shape == (n, l, 2)
        assert np.isclose(np.sum(G * XE), np.sum(adj * E), rtol=1e-10)
    one = O.rtsvd_adjoint(out, G[:, :, 1:2])
    assert np.allclose(adj[:, :, 1:2], one, rtol=0, atol=1e-12 * np.abs(one).max())


def test_ttsvd_adjoint_satisfies_the_adjoint_identity():
    """<G, X_s(E)> = <adjoint(G), E> with X_s(E) from ttsvd_solve itself at
    the chosen s, and at full rank the adjoint of B -> A^{-1} * B is
    A^{-T} * G (the t-transpose of the inverse)."""
    A, B, delta = small_blur_multi(p=2)
    n, l, m = A.shape
    out = O.ttsvd_solve(A, B, delta, 1.1)
    g = np.random.default_rng(78)
    for _ in range(3):
        E = g.standard_normal((n, l, 2))
        G = g.standard_normal((n, m, 2))
        XE = O.ttsvd_solve(A, E, delta, 1.1, k_fixed=out["k"])["X"]
        assert np.isclose(np.sum(G * XE), np.sum(O.ttsvd_adjoint(A, out, G) * E), rtol=1e-10)
    full = dict(out, k=min(l, m))
    G = g.standard_normal((n, m, 1))
    Ainv = O.ifft3_real(np.linalg.inv(O.fft3(A)))
    want = O.tprod_bcirc(O.ttranspose(Ainv), G)
    assert np.allclose(O.ttsvd_adjoint(A, full, G), want, rtol=0, atol=1e-9 * np.abs(want).max())


def test_ttsvd_discrepancy_bracket_with_brute_force_residual():
    A, B, delta = small_blur()
    tau = 1.1
    out = O.ttsvd_solve(A, B, delta, tau)
    k = out["k"]
    r = lambda X: np.sqrt(O.fro2(B - O.tprod_bcirc(A, X)))
    assert r(out["X"]) <= tau * delta * (1 + 1e-12)
    if k > 1:
        assert r(O.ttsvd_solve(A, B, delta, tau, k_fixed=k - 1)["X"]) > tau * delta
    assert np.isclose(r(out["X"]), out["res"][k], rtol=1e-8)


# ------------------------------------------------------------ tGKB ----

def test_tgkb_decomposition_orthonormality_and_start():
    n, l, m, k = 6, 9, 7, 4
    A = rnd((n, l, m), 8)
    B = rnd((n, l, 1), 9)
    g = O.tgkb_hat(O.fft3(A), O.fft3(B)[:, :, 0], k)
    W = spatial(g["W"])
    Q = spatial(g["Q"])
    # bidiagonal tensor P_k: tubes c_i on the diagonal and z_{i+1} below
    Ph = np.zeros((n, k + 1, k), complex)
    for s in range(n):
        Ph[s] = O.bidiag(g["c"][s], g["z"][s], k)
    P = spatial(Ph)
    assert np.allclose(O.tprod_bcirc(A, W), O.tprod_bcirc(Q, P), atol=1e-10)      # Eq. (t-gkb)
    assert np.allclose(O.tprod_bcirc(O.ttranspose(W), W), O.tidentity(k, n), atol=1e-10)
    assert np.allclose(O.tprod_bcirc(O.ttranspose(Q), Q), O.tidentity(k + 1, n), atol=1e-10)
    z1 = spatial(g["z"][:, 0].astype(complex)[:, None, None])
    e1z1 = np.zeros((n, k + 1, 1))
    e1z1[:, 0, 0] = z1[:, 0, 0]
    assert np.allclose(O.tprod_bcirc(O.ttranspose(Q), B), e1z1, atol=1e-10)       # Q^T * B = e1 * z1
    assert np.all(g["c"] >= 0) and np.all(g["z"] >= 0)


@pytest.mark.parametrize("k", [1, 2, 4])
def test_tgkb_solution_is_the_krylov_least_squares_solution(k):
    """Per Fourier slice, X_k minimises ||b - A x|| over the Krylov space
    K_k(A^H A, A^H b) (Eq. (krylov1)), here built from explicit power vectors."""
    A, B, delta = small_blur(N=9, n=5, general=0.3)
    out = O.tgkb_solve(A, B, delta, 1.1, 50, k_fixed=k)
    Ah, Bh = O.fft3(A), O.fft3(B)
    Xh = np.zeros((A.shape[0], A.shape[2], 1), complex)
    for s in range(A.shape[0]):
        M, b = Ah[s], Bh[s, :, 0]
        v = M.conj().T @ b
        K = [v]
        for _ in range(k - 1):
            v = M.conj().T @ (M @ v)
            K.append(v)
        Kq, _ = np.linalg.qr(np.stack(K, axis=1))
        y, *_ = np.linalg.lstsq(M @ Kq, b, rcond=None)
        Xh[s, :, 0] = Kq @ y
    assert np.allclose(out["X"], spatial(Xh), atol=1e-8 * np.abs(out["X"]).max())


@pytest.mark.parametrize("k", [1, 2, 4])
def test_tgkb_solution_is_the_cgls_iterate(k):
    """Per Fourier slice, X_k is the k-th iterate of textbook CGLS on
    (A-hat_s, b-hat_s) from x = 0 (the same Krylov least-squares problem,
    reached by a different recurrence: short-term, no reorthogonalisation)."""
    A, B, delta = small_blur(N=9, n=5, general=0.3)
    out = O.tgkb_solve(A, B, delta, 1.1, 50, k_fixed=k)
    Ah, Bh = O.fft3(A), O.fft3(B)
    Xh = np.zeros((A.shape[0], A.shape[2], 1), complex)
    for s in range(A.shape[0]):
        M, b = Ah[s], Bh[s, :, 0]
        x = np.zeros(M.shape[1], complex)
        r = b.copy()
        g = M.conj().T @ r
        d = g.copy()
        gg = np.vdot(g, g).real
        for _ in range(k):
            q = M @ d
            alpha = gg / np.vdot(q, q).real
            x = x + alpha * d
            r = r - alpha * q
            g = M.conj().T @ r
            gg_new = np.vdot(g, g).real
            d = g + (gg_new / gg) * d
            gg = gg_new
        Xh[s, :, 0] = x
    assert np.allclose(out["X"], spatial(Xh), atol=1e-8 * np.abs(out["X"]).max())


def test_tgkb_full_space_solves_the_system():
    n, m = 4, 5
    A = rnd((n, m, m), 10) + 3 * O.tidentity(m, n)
    X = rnd((n, m, 1), 11)
    B = O.tprod_bcirc(A, X)
    out = O.tgkb_solve(A, B, 1e-14, 1.1, m, k_fixed=m)
    assert np.allclose(out["X"], X, atol=1e-9)


def test_tgkb_discrepancy_bracket_with_brute_force_residual():
    A, B, delta = small_blur()
    tau = 1.1
    out = O.tgkb_solve(A, B, delta, tau, 20)
    k = out["k"]
    assert out["status"] == O.STATUS_OK
    r = lambda X: np.sqrt(O.fro2(B - O.tprod_bcirc(A, X)))
    assert np.isclose(r(out["X"]), out["res"][k], rtol=1e-8)
    assert out["res"][k] <= tau * delta
    if k > 1:
        assert r(O.tgkb_solve(A, B, delta, tau, 20, k_fixed=k - 1)["X"]) > tau * delta


def test_ritz_triplets_relations_and_full_rank_limit():
    """Section 4.3's triplets from k tGKB steps: A-hat V_i = U_i s_i exactly in
    every Fourier slice (from A W_k = Q_{k+1} P_k), orthonormal U and V; the
    tGKB solution rebuilt from them (Eq. (solgkbb)) is the tGKB solution; and
    with k = min(l, m) the singular values are those of the full tSVD."""
    A, B, delta = small_blur(N=10, n=6, general=0.05)
    n, l, m = A.shape
    k = 5
    t = O.ritz_triplets(A, B, k)
    Ah = O.fft3(A)
    for s in range(n):
        assert np.allclose(Ah[s] @ t["Vh"][s], t["Uh"][s] * t["S"][s][None, :], atol=1e-10)
        assert np.allclose(t["Uh"][s].conj().T @ t["Uh"][s], np.eye(k), atol=1e-10)
        assert np.allclose(t["Vh"][s].conj().T @ t["Vh"][s], np.eye(k), atol=1e-10)
    Bh = O.fft3(B)
    Xh = np.stack([t["Vh"][s] @ ((t["Uh"][s].conj().T @ Bh[s]) / t["S"][s][:, None]) for s in range(n)])
    ref = O.tgkb_solve(A, B, delta, 1.1, k, k_fixed=k)["X"]
    assert np.allclose(O.ifft3_real(Xh), ref, atol=1e-10 * np.abs(ref).max())
    full = O.ritz_triplets(A, B, min(l, m))
    _, S_exact, _ = O.tsvd_hat(Ah)
    assert np.allclose(full["S"], S_exact[:, :min(l, m)], rtol=1e-8, atol=1e-12)


def slice_noise(A, Xt, levels, seed):
    """B = A*Xt + E with slice j's noise of relative level levels[j];
    returns B and delta_j = ||E_j||_F."""
    Bt = O.tprod_bcirc(A, Xt)
    g = np.random.default_rng(seed)
    B, deltas = Bt.copy(), []
    for j, lev in enumerate(levels):
        E = g.standard_normal(Bt[:, :, j].shape)
        E = lev * E / np.linalg.norm(E) * np.linalg.norm(Bt[:, :, j])
        B[:, :, j] += E
        deltas.append(float(np.linalg.norm(E)))
    return B, deltas


def test_tgkb_p_each_slice_meets_its_own_discrepancy_bound():
    """tGKB_p (problem (I6) with ||E_j|| <= delta_j): slice j stops at the
    first k_j whose residual ||B_j - A*X_j||_F, formed here through the
    block-circulant product, is <= tau delta_j; different noise levels give
    different k_j."""
    A, _, _ = small_blur_multi(p=3)
    Xt = np.concatenate([synth.lateral(synth.synthetic_image(10, 8, 3, 1, np.random.default_rng(40 + j)))
                         for j in range(3)], axis=2)
    B, deltas = slice_noise(A, Xt, [1e-1, 1e-2, 1e-3], 41)
    tau = 1.1
    out = O.tgkb_p_solve(A, B, deltas, tau, 10)
    assert out["X"].shape == (8, 10, 3)
    r = lambda X, j: np.sqrt(O.fro2(B[:, :, j:j + 1] - O.tprod_bcirc(A, X)))
    for j in range(3):
        kj = out["k"][j]
        assert out["status"][j] == O.STATUS_OK
        assert r(out["X"][:, :, j:j + 1], j) <= tau * deltas[j] * (1 + 1e-12)
        if kj > 1:
            prev = O.tgkb_solve(A, B[:, :, j:j + 1], deltas[j], tau, 10, k_fixed=kj - 1)["X"]
            assert r(prev, j) > tau * deltas[j]
    assert out["k"][0] < out["k"][1] < out["k"][2]


def test_tgkb_p_slices_are_independent_and_homogeneous():
    """Changing one slice leaves the others' k_j and X_j alone; scaling B_j
    and delta_j by a > 0 scales X_j by a with the same k_j (the method is
    positively homogeneous: Normalize divides the scale out)."""
    A, B, delta = small_blur_multi(p=3)
    d = [delta / np.sqrt(3.0)] * 3
    tau = 1.1
    out = O.tgkb_p_solve(A, B, d, tau, 10)
    B2 = B.copy()
    B2[:, :, 2] = 3.0 * B[:, :, 2] + 0.5
    out2 = O.tgkb_p_solve(A, B2, [d[0], d[1], 3.0 * d[2]], tau, 10)
    for j in range(2):
        assert out2["k"][j] == out["k"][j]
        assert np.array_equal(out2["X"][:, :, j], out["X"][:, :, j])
    B3 = B.copy()
    B3[:, :, 1] *= 7.5
    out3 = O.tgkb_p_solve(A, B3, [d[0], 7.5 * d[1], d[2]], tau, 10)
    assert out3["k"] == out["k"]
    assert np.allclose(out3["X"][:, :, 1], 7.5 * out["X"][:, :, 1], rtol=0, atol=1e-11 * np.abs(out3["X"]).max())


def test_nested_tgkb_p_first_slice_is_tgkb_and_residuals_split():
    """Algorithm 6: slice 1 is the tGKB solution at its k (a different code
    path: Q_{k+1}^T * B_1 = e_1 z_1 there); every slice's true residual splits
    into the tested projected residual and the part of B_j outside the span
    of Q_{k+1} (Pythagoras, both sides brute force through the block-circulant
    product); k never decreases and starts at k_init = 2."""
    A, B, delta = small_blur_multi(p=3)
    d = [delta / np.sqrt(3.0)] * 3
    eta = 1.1
    out = O.nested_tgkb_p_solve(A, B, d, eta, 10)
    k = out["k"]
    assert k == sorted(k) and k[0] >= 2 and all(st == O.STATUS_OK for st in out["status"])
    x1 = O.tgkb_solve(A, B[:, :, :1], d[0], eta, 10, k_fixed=k[0])["X"]
    assert np.allclose(out["X"][:, :, :1], x1, rtol=0, atol=1e-10 * np.abs(x1).max())
    n = A.shape[0]
    for j in range(3):
        kj = k[j]
        Qh = out["Q"][:, :, :kj + 1]
        bh = O.fft3(B[:, :, j:j + 1])[:, :, 0]
        outside = O.ifft3_real((bh - np.einsum("sdi,si->sd", Qh, np.einsum("sdi,sd->si", np.conj(Qh), bh)))[:, :, None])
        true2 = O.fro2(B[:, :, j:j + 1] - O.tprod_bcirc(A, out["X"][:, :, j:j + 1]))
        assert np.isclose(true2, out["res"][j][kj] ** 2 + O.fro2(outside), rtol=1e-9)
        assert out["res"][j][kj] < eta * d[j]


def test_nested_tgkb_p_duplicate_and_loose_slices_do_not_grow_the_basis():
    """A repeated slice with the same bound reuses k and gives the same
    solution; a slice whose bound is already met keeps k unchanged."""
    A, B, delta = small_blur_multi(p=2)
    d0 = delta / np.sqrt(2.0)
    Bd = np.concatenate([B[:, :, :1], B[:, :, :1], B[:, :, 1:2]], axis=2)
    out = O.nested_tgkb_p_solve(A, Bd, [d0, d0, 1e6], 1.1, 10)
    assert out["k"][1] == out["k"][0] == out["k"][2]
    assert np.allclose(out["X"][:, :, 1], out["X"][:, :, 0], rtol=0, atol=1e-12 * np.abs(out["X"]).max())


# ------------------------------------------------------------ tGKT ----

def test_tgkt_full_space_is_dense_tikhonov():
    A, B, delta = small_blur(N=6, n=4, general=0.2)
    n, l, m = A.shape
    g = O.tgkb_solve(A, B, delta, 1.1, m, k_fixed=m)
    Ah, Bh = O.fft3(A), O.fft3(B)
    for mu in [0.3, 10.0, 1e3]:
        X, _ = O.tikhonov_fixed_mu(g, mu)
        Xh = np.zeros((n, m, 1), complex)
        for s in range(n):
            M = Ah[s]
            Xh[s] = np.linalg.solve(M.conj().T @ M + np.eye(m) / mu, M.conj().T @ Bh[s])
        assert np.allclose(X, spatial(Xh), atol=1e-8 * np.abs(X).max())


def test_tgkt_residual_monotone_limit_and_root():
    A, B, delta = small_blur()
    tau = 1.1
    out = O.tgkt_solve(A, B, delta, tau, 20, 1e-3, 1e9)
    g = out["gkb"]
    mus = np.logspace(-3, 9, 25)
    res = [O.tikhonov_fixed_mu(g, mu)[1] for mu in mus]
    assert all(res[i + 1] <= res[i] * (1 + 1e-12) for i in range(len(res) - 1))
    X_inf, _ = O.tikhonov_fixed_mu(g, 1e14)
    assert np.allclose(X_inf, g["X"], atol=1e-6 * np.abs(g["X"]).max())
    assert out["status"] == O.STATUS_OK
    assert np.isclose(out["residual"], tau * delta, rtol=1e-9)
    # the residual reported is the true ||B - A * X_mu|| of the returned solution
    assert np.isclose(np.sqrt(O.fro2(B - O.tprod_bcirc(A, out["X"]))), out["residual"], rtol=1e-7)


def test_tgkt_adjoint_matches_central_differences_on_64_directions():
    """dL/dB of the Tikhonov-tGKB solution at fixed k and mu (the reverse
    sweep through Algorithm 4) against FP64 central differences of the
    forward map, L = ||X - X_true||_F^2, on 64 seeded directions."""
    A, B, _ = small_blur(N=10, n=8, general=0.02)
    k, mu = 5, 300.0
    g = np.random.default_rng(41)
    Xt = g.standard_normal((8, 10, 1))
    X = O.tgkt_fixed(A, B, k, mu)
    dB, Xa = O.tgkt_adjoint(A, B, k, mu, 2.0 * (X - Xt))
    assert np.allclose(Xa, X, atol=1e-13 * np.abs(X).max())
    loss = lambda Bv: float(np.sum((O.tgkt_fixed(A, Bv, k, mu) - Xt) ** 2))
    h = 1e-6
    for _ in range(64):
        D = g.standard_normal(B.shape)
        D *= np.linalg.norm(B) / np.linalg.norm(D)
        fd = (loss(B + h * D) - loss(B - h * D)) / (2 * h)
        assert abs(fd - np.sum(dB * D)) <= 1e-7 * np.linalg.norm(dB) * np.linalg.norm(D)


def test_tgkt_adjoint_at_infinite_mu_is_the_tgkb_adjoint():
    """mu = inf (no damping) gives the tGKB solution of Eq. (solgkb) at k
    steps, and the reverse sweep its dL/dB: the forward against tgkb_solve,
    the gradient against central differences on 64 seeded directions."""
    A, B, _ = small_blur(N=10, n=8, general=0.02)
    k = 4
    X = O.tgkb_solve(A, B, 0.0, 1.0, k, k_fixed=k)["X"]
    g = np.random.default_rng(43)
    W = g.standard_normal(X.shape)
    dB, Xa = O.tgkt_adjoint(A, B, k, np.inf, W)
    assert np.allclose(Xa, X, atol=1e-12 * np.abs(X).max())
    loss = lambda Bv: float(np.sum(W * O.tgkb_solve(A, Bv, 0.0, 1.0, k, k_fixed=k)["X"]))
    h = 1e-6
    for _ in range(64):
        D = g.standard_normal(B.shape)
        D *= np.linalg.norm(B) / np.linalg.norm(D)
        fd = (loss(B + h * D) - loss(B - h * D)) / (2 * h)
        assert abs(fd - np.sum(dB * D)) <= 1e-7 * np.linalg.norm(dB) * np.linalg.norm(D)


def test_tgkt_adjoint_on_the_full_space_is_the_dense_tikhonov_adjoint():
    """With k = m the Krylov space is all of C^m and the solution is the dense
    Tikhonov solution X-hat_s = (A_s^H A_s + I/mu)^{-1} A_s^H B-hat_s, linear in
    B: its adjoint applied to G is A_s (A_s^H A_s + I/mu)^{-1} G-hat_s per
    slice (the subspace terms of the reverse sweep must cancel)."""
    A, B, _ = small_blur(N=6, n=4, general=0.2)
    n, l, m = A.shape
    mu = 20.0
    G = rnd((n, m, 1), 42)
    dB, _ = O.tgkt_adjoint(A, B, m, mu, G)
    Ah, Gh = O.fft3(A), O.fft3(G)
    Yh = np.zeros((n, l, 1), complex)
    for s in range(n):
        M = Ah[s]
        Yh[s] = M @ np.linalg.solve(M.conj().T @ M + np.eye(m) / mu, Gh[s])
    assert np.allclose(dB, spatial(Yh), atol=1e-8 * np.abs(dB).max())


# ---------------------------------------------------------- t-Lanczos ----

def test_tlanczos_decomposition_on_a_symmetric_tensor():
    n, m, k = 5, 7, 3
    M = rnd((n, m, m), 12)
    A = O.tprod(O.ttranspose(M), M)                # t-symmetric: A^T = A
    assert np.allclose(O.ttranspose(A), A, atol=1e-12)
    B = rnd((n, m, 1), 13)
    g = O.tlanczos_hat(O.fft3(A), O.fft3(B)[:, :, 0], k)
    Q = spatial(g["Q"])
    Th = np.stack([O.tridiag(g["c"][s], g["z"][s], k) for s in range(n)])
    T = spatial(Th)
    assert np.allclose(O.tprod_bcirc(A, Q[:, :, :k]), O.tprod_bcirc(Q, T), atol=1e-9)   # Eq. (t-lanczos)
    assert np.allclose(O.tprod_bcirc(O.ttranspose(Q), Q), O.tidentity(k + 1, n), atol=1e-9)


def test_tlanczos_method_meets_the_discrepancy_principle():
    n, m = 6, 8
    M = rnd((n, m, m), 14)
    A = O.tprod(O.ttranspose(M), M) + 0.5 * O.tidentity(m, n)
    X = rnd((n, m, 1), 15)
    B = O.tprod(A, X)
    E = rnd(B.shape, 16)
    E = 1e-2 * E / np.linalg.norm(E) * np.linalg.norm(B)
    out = O.tlanczos_solve(A, B + E, np.linalg.norm(E), 1.1, m)
    assert out["status"] == O.STATUS_OK
    assert np.sqrt(O.fro2(B + E - O.tprod_bcirc(A, out["X"]))) <= 1.1 * np.linalg.norm(E) * (1 + 1e-9)


# ------------------------------------------- small end-to-end workload ----

def test_small_workload_end_to_end():
    P = synth.blur_problem("n32")
    cfg = P["cfg"]
    A, B, Om = (P[k].astype(np.float64) for k in ("A", "B", "Omega"))
    Xt = P["X_true"].astype(np.float64)
    err = lambda X: np.linalg.norm(X - Xt) / np.linalg.norm(Xt)
    t = O.ttsvd_solve(A, B, P["delta"], cfg.tau)
    r = O.rtsvd_solve(A, B, Om, P["delta"], cfg.tau, cfg.eps_rel * P["norm_A"], cfg.p_over,
                      cfg.block, cfg.q_power, cfg.r_max)
    g = O.tgkb_solve(A, B, P["delta"], cfg.tau, cfg.k_max)
    tk = O.tgkt_solve(A, B, P["delta"], cfg.tau, cfg.k_max, cfg.mu_lo, cfg.mu_hi)
    for out in (t, r, g, tk):
        assert out["status"] == O.STATUS_OK
        assert err(out["X"]) < 0.3
    # the qualitative findings of Section 5's tables on this synthetic workload
    assert g["k"] < t["k"]                  # tGKB needs fewer steps than T-tSVD's k
    assert r["r"] - cfg.p_over <= r["k"] < r["r"]   # RT-tSVD at or just above k_init = r - rho (Table 0's rows)
    assert abs(err(r["X"]) - err(t["X"])) < 0.01 * err(t["X"])   # RT-tSVD as accurate as T-tSVD
    assert err(tk["X"]) <= err(g["X"])      # the Tikhonov variant at least as accurate as tGKB


def test_zero_right_hand_side_gives_the_zero_solution():
    """B = 0: Normalize breaks down on every slice (zero vector substitute),
    the residual is 0 at the first admissible k, and X = 0 exactly."""
    A, B, delta = small_blur()
    n, l, m = A.shape
    Z = np.zeros_like(B)
    Om = rnd((n, m, m), 30)
    eps = 0.02 * np.sqrt(O.fro2(A))
    g = O.tgkb_solve(A, Z, delta, 1.1, 6)
    r = O.rtsvd_solve(A, Z, Om, delta, 1.1, eps, 3, 2, 1, r_max=m)
    t = O.ttsvd_solve(A, Z, delta, 1.1)
    k = O.tgkt_solve(A, Z, delta, 1.1, 6, 1e-3, 1e5)
    assert (g["k"], t["k"], k["k"]) == (1, 1, 1) and r["k"] == max(1, r["r"] - 3)
    for o in (g, r, t, k):
        assert o["status"] == O.STATUS_OK
        assert not np.any(o["X"])


def test_zero_delta_runs_to_the_cap():
    """delta = 0: the discrepancy bound is 0, so the iterative methods stop at
    their caps with NOT_CONVERGED, while the T-tSVD reaches full rank, where
    the residual of a square nonsingular A is exactly 0 (captured energy
    clamped at ||B||^2)."""
    A, B, delta = small_blur()
    n, l, m = A.shape
    Om = rnd((n, m, m), 31)
    eps = 0.02 * np.sqrt(O.fro2(A))
    g = O.tgkb_solve(A, B, 0.0, 1.1, 6)
    r = O.rtsvd_solve(A, B, Om, 0.0, 1.1, eps, 3, 2, 1, r_max=m)
    k = O.tgkt_solve(A, B, 0.0, 1.1, 6, 1e-3, 1e5)
    t = O.ttsvd_solve(A, B, 0.0, 1.1)
    assert g["k"] == 6 and g["status"] == O.STATUS_NOT_CONVERGED
    assert r["k"] == r["r"] and r["status"] == O.STATUS_NOT_CONVERGED
    assert k["status"] == O.STATUS_NOT_CONVERGED and k["mu"] == 1e5
    assert t["k"] == min(l, m) and t["status"] == O.STATUS_OK
    assert np.isclose(np.sqrt(O.fro2(B - O.tprod(A, t["X"]))), 0.0, atol=1e-10 * np.sqrt(O.fro2(B)))


def test_uneven_batch_carries_a_calibrated_tolerance_per_problem():
    """The bench's uneven batch: every problem has r_max = min(N, 160) and the
    eps_rel its calibration chose (synth.UNEVEN_EPS_J, written from
    tests/golden/calibrate_eps.py); a smaller or reseeded batch has none."""
    probs = synth.uneven_problems()
    assert len(probs) == 16 and len(synth.UNEVEN_EPS_J) == 16
    for p, j in zip(probs, synth.UNEVEN_EPS_J):
        assert p["r_max"] == min(p["N"], 160)
        assert p["eps_rel"] == 10.0 ** (-j / 10.0)
    assert all(p["eps_rel"] is None for p in synth.uneven_problems(count=3))
