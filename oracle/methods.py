"""FP64 oracle, part 2: the regularised solvers (Sections 1, 3.2, 4 and 5).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every method works per Fourier frontal slice on the full spectrum of n slices,
the way the paper's algorithms loop over i = 1..n.  Slices are coupled only
through Frobenius norms (Parseval: ||X||_F^2 = (1/n) sum_s ||Xh[s]||^2) and the
shared truncation index.

Readings of points the paper leaves open (each also listed in the design notes):
  * Eq. (disp): the residual is ||B - A * X_k||_F with the true A, and k is
    the smallest admissible index with residual <= tau * delta.
  * Eq. (kinit): for RT-tSVD the admissible k run from max(1, r - p) to r;
    T-tSVD, tGKB and t-Lanczos start at k = 1.  If no admissible k meets the
    bound the last one is returned with status NOT_CONVERGED.
  * s_j^{-1} in Eq. (14) and its RT-tSVD analogue: a singular value at or
    below max(l, m) * eps * sigma_max (sigma_max over all slices) is treated
    as zero (its term is dropped), the usual numerical-rank convention.
  * Algorithm 3 is run in block form: b Gaussian slices at a time, q power
    iterations, each block orthonormalised by two classical Gram-Schmidt
    passes against the basis so far and then column by column (two passes and
    a Normalize per column).  With b = 1, q = 0 this reduces to Algorithm 3
    (pinned in the tests against rtsvd_alg3, which follows Algorithm 3 as
    printed).  The indicator eta and its stopping rule are Algorithm 3's.
  * Algorithm 4's reorthogonalisation steps use two classical Gram-Schmidt
    passes.
  * tGKT: the projected Tikhonov problem min ||P_k y - z_1 e_1||^2 + mu^{-1}||y||^2
    per slice, one scalar mu for all slices, mu found by bisection on log10(mu)
    over the interval of Section 5 so that the residual equals tau * delta.
"""
from __future__ import annotations

import numpy as np

from .talgebra import fft3, ifft3_real, fro2, fro2_hat, normalize_hat, tsvd_hat

STATUS_OK = 0
STATUS_NOT_CONVERGED = -5

EPS64 = float(np.finfo(np.float64).eps)


def _ct(M: np.ndarray) -> np.ndarray:
    """Conjugate transpose of every slice of a stacked (n, a, b) array."""
    return np.conj(np.swapaxes(M, -1, -2))


def _dp_pick(res: dict, tau_delta: float, k_lo: int, k_hi: int):
    """Smallest k in [k_lo, k_hi] with res[k] <= tau*delta (Eq. (disp))."""
    for k in range(k_lo, k_hi + 1):
        if res[k] <= tau_delta:
            return k, STATUS_OK
    return k_hi, STATUS_NOT_CONVERGED


def _margin(res: dict, k: int, tau_delta: float) -> float:
    """Relative distance of the DP test from a tie at the chosen k and at k-1.
    With delta = 0 the bound tau*delta is 0: residuals are compared with 0
    exactly, so the margin is infinite unless a residual is exactly 0."""
    vals = [abs(res[k] - tau_delta)]
    if (k - 1) in res:
        vals.append(abs(res[k - 1] - tau_delta))
    if tau_delta == 0.0:
        return float("inf") if min(vals) > 0.0 else 0.0
    return float(min(vals) / tau_delta)


def _inv_sigma(S: np.ndarray, dims: int) -> np.ndarray:
    """1/sigma with the numerical-rank threshold max(l,m) * eps * sigma_max."""
    tol = dims * EPS64 * (float(S.max()) if S.size else 0.0)
    out = np.zeros_like(S)
    keep = S > tol
    out[keep] = 1.0 / S[keep]
    return out


# --------------------------------------------------------------------------
# T-tSVD method (Section 4.1, Eqs. (11)-(14)).
# --------------------------------------------------------------------------

def ttsvd_solve(A, B, delta, tau, k_fixed=None):
    n, l, m = A.shape
    Ah, Bh = fft3(A), fft3(B)
    U, S, V = tsvd_hat(Ah)
    qn = S.shape[1]
    beta = _ct(U) @ Bh                                   # (n, q, p)
    b2 = np.sum(np.abs(Bh) ** 2)
    captured = np.concatenate([[0.0], np.cumsum(np.sum(np.abs(beta) ** 2, axis=(0, 2)))])
    res = {k: float(np.sqrt(max(b2 - captured[k], 0.0) / n)) for k in range(qn + 1)}
    td = tau * delta
    k, status = _dp_pick(res, td, 1, qn)
    if k_fixed is not None:
        k, status = k_fixed, STATUS_OK
    alpha = _inv_sigma(S, max(l, m))[:, :, None] * beta
    Xh = V[:, :, :k] @ alpha[:, :k, :]
    return dict(X=ifft3_real(Xh), k=k, status=status, res=res, tau_delta=td,
                margin=_margin(res, k, td), S=S)


def ttsvd_adjoint(A, out: dict, G: np.ndarray) -> np.ndarray:
    """Adjoint of the linear map B -> X_s of a ttsvd_solve result at its s:
    X_s = V_s S_s^{-1} U_s^T * B (Eq. (14)), so dL/dB = U_s S_s^{-1} V_s^T * G,
    slice by slice from the full tSVD of A; singular values the solve dropped
    (_inv_sigma) are dropped here too."""
    n, l, m = A.shape
    k = out["k"]
    U, S, V = tsvd_hat(fft3(A))
    inv = _inv_sigma(S, max(l, m))[:, :k]
    t = _ct(V[:, :, :k]) @ fft3(G)
    return ifft3_real(U[:, :, :k] @ (inv[:, :, None] * t))


# --------------------------------------------------------------------------
# R-tSVD, Algorithm 3 exactly as printed (one Gaussian slice per step).
# --------------------------------------------------------------------------

def rtsvd_alg3(A, Omega, eps, r_max=None):
    """Algorithm 3: grows Q one lateral slice at a time until eta < eps^2.

    Omega[:, :, r-1] (spatial, m x 1 x n) is the Gaussian slice G drawn at
    step r.  Returns Fourier-domain Q (n, l, r), Bt (n, r, m), r, eta history.
    """
    n, l, m = A.shape
    r_max = m if r_max is None else r_max
    Ah = fft3(A)
    eta = fro2(A)
    etas = [eta]
    Q, Bt = [], []
    r = 0
    while eta >= eps * eps and r < r_max:
        r += 1
        Gh = fft3(Omega[:, :, r - 1])                    # (n, m)
        Zh = np.einsum("sij,sj->si", Ah, Gh)             # A * G
        if r > 1:                                        # - Q_{r-1} * (Bt(r-1,:,:) * G)
            tube = np.einsum("sj,sj->s", Bt[-1], Gh)
            Zh = Zh - Q[-1] * tube[:, None]
        Zh, _ = normalize_hat(Zh)
        if r > 1:                                        # Z - sum_j Q_j * (Q_j^T * Z)
            coef = [np.einsum("si,si->s", np.conj(Qj), Zh) for Qj in Q]
            for Qj, cj in zip(Q, coef):
                Zh = Zh - Qj * cj[:, None]
        Zh, _ = normalize_hat(Zh)
        Q.append(Zh)
        Y = np.einsum("si,sij->sj", np.conj(Zh), Ah)     # Y = Z^T * A
        Bt.append(Y)
        eta = eta - fro2_hat(Y)
        etas.append(eta)
    Qa = np.stack(Q, axis=2) if Q else np.zeros((n, l, 0), complex)
    Ba = np.stack(Bt, axis=1) if Bt else np.zeros((n, 0, m), complex)
    return dict(Q=Qa, Bt=Ba, r=r, eta=eta, etas=etas)


def _orth_block(Y: np.ndarray, Q: np.ndarray | None) -> np.ndarray:
    """Two CGS passes of Y against Q, then column-by-column CGS2 + Normalize."""
    Y = np.array(Y, dtype=np.complex128, copy=True)
    if Q is not None and Q.shape[2] > 0:
        QH = _ct(Q)
        for _ in range(2):
            Y = Y - Q @ (QH @ Y)
    b = Y.shape[2]
    for j in range(b):
        if j > 0:
            P = Y[:, :, :j]
            PH = _ct(P)
            for _ in range(2):
                Y[:, :, j:j + 1] = Y[:, :, j:j + 1] - P @ (PH @ Y[:, :, j:j + 1])
        Y[:, :, j], _ = normalize_hat(Y[:, :, j])
    return Y


def rtsvd_block(A, Omega, eps, b, q, r_max):
    """Block form of Algorithm 3 with q power iterations (see module notes).

    Returns Fourier-domain Q (n, l, r), BH = Bt^H (n, m, r), r, eta history.
    """
    n, l, m = A.shape
    Ah = fft3(A)
    AhH = _ct(Ah)
    eta = fro2(A)
    etas = [eta]
    Q = np.zeros((n, l, 0), complex)
    BH = np.zeros((n, m, 0), complex)
    r = 0
    while eta >= eps * eps and r < r_max:
        bb = min(b, r_max - r)
        Gh = fft3(Omega[:, :, r:r + bb])
        Y = _orth_block(Ah @ Gh, Q)
        for _ in range(q):
            Z = _orth_block(AhH @ Y, None)
            Y = _orth_block(Ah @ Z, Q)
        BHb = AhH @ Y
        eta = eta - fro2_hat(BHb)
        etas.append(eta)
        Q = np.concatenate([Q, Y], axis=2)
        BH = np.concatenate([BH, BHb], axis=2)
        r += bb
    return dict(Q=Q, Bt=_ct(BH), r=r, eta=eta, etas=etas)


# --------------------------------------------------------------------------
# RT-tSVD method (Section 4.2 and Eq. (kinit)).
# --------------------------------------------------------------------------

def rtsvd_prefix(fac: dict, r: int, block: int) -> dict:
    """The block-form factorisation stopped after its first r columns (r a
    multiple of the block size, or the full r): the blocks are built one after
    another, so this is what rtsvd_block returns when eta falls below eps^2
    right after column r."""
    nb = -(-r // block)
    return dict(Q=fac["Q"][:, :, :r], Bt=fac["Bt"][:, :r, :], r=r, eta=fac["etas"][nb], etas=fac["etas"][:nb + 1])


def rtsvd_solve(A, B, Omega, delta, tau, eps, p_over, block=16, q_power=1,
                r_max=None, form="block", k_fixed=None, fac=None):
    n, l, m = A.shape
    r_max = min(l, m) if r_max is None else r_max
    if fac is not None:
        pass  # a factorisation made earlier (rtsvd_block / rtsvd_prefix) with this eps
    elif form == "alg3":
        fac = rtsvd_alg3(A, Omega, eps, r_max)
    else:
        fac = rtsvd_block(A, Omega, eps, block, q_power, r_max)
    Q, Bt, r = fac["Q"], fac["Bt"], fac["r"]
    Ah, Bh = fft3(A), fft3(B)
    Ub, S, V = tsvd_hat(Bt)                               # full tSVD of Bt
    d = _ct(Q) @ Bh                                       # (n, r, p)
    beta = _ct(Ub) @ d                                    # U_k^T * B in Fourier
    alpha = _inv_sigma(S, max(l, m))[:, :, None] * beta
    k_init = max(1, r - p_over)
    td = tau * delta
    res = {}
    for k in range(k_init, r + 1):
        Xh = V[:, :, :k] @ alpha[:, :k, :]
        res[k] = float(np.sqrt(fro2_hat(Bh - Ah @ Xh)))
    k, status = _dp_pick(res, td, k_init, r)
    if fac["eta"] >= eps * eps:
        status = STATUS_NOT_CONVERGED
    if k_fixed is not None:
        k, status = k_fixed, STATUS_OK
    Xh = V[:, :, :k] @ alpha[:, :k, :]
    return dict(X=ifft3_real(Xh), k=k, r=r, k_init=k_init, status=status, res=res,
                tau_delta=td, margin=_margin(res, k, td), eta=fac["eta"],
                etas=fac["etas"], S=S, Q=Q, Bt=Bt)


# --------------------------------------------------------------------------
# tGKB (Algorithm 4) and the tGKB method (Eqs. (9tt), (solgkb)).
# --------------------------------------------------------------------------

def rtsvd_adjoint(out: dict, G: np.ndarray) -> np.ndarray:
    """Adjoint of the linear map B -> X_k of an rtsvd_solve result, at its k:
    X_k = V_k S_k^{-1} U_k^T * B (Section 4.2, with U_k = Q * U-tilde_k from the
    full tSVD of B-tilde), so dL/dB = U_k S_k^{-1} V_k^T * G for G = dL/dX_k,
    the t-transpose of the filter (Section 2: the t-product's adjoint is the
    t-transpose).  Fourier slice by slice; singular values the solve dropped
    (_inv_sigma) are dropped here too."""
    Q, Bt, k = out["Q"], out["Bt"], out["k"]
    Ub, S, V = tsvd_hat(Bt)
    l, m = Q.shape[1], V.shape[1]
    inv = _inv_sigma(S, max(l, m))[:, :k]
    Uk = Q @ Ub[:, :, :k]                                 # (n, l, k)
    t = _ct(V[:, :, :k]) @ fft3(G)                        # (n, k, p)
    return ifft3_real(Uk @ (inv[:, :, None] * t))


def _reorth(v: np.ndarray, basis: list) -> np.ndarray:
    """Two CGS passes of v (n, d) against the Fourier-domain vectors in basis."""
    if not basis:
        return v
    Bm = np.stack(basis, axis=2)                          # (n, d, j)
    for _ in range(2):
        coef = np.einsum("sdj,sd->sj", np.conj(Bm), v)
        v = v - np.einsum("sdj,sj->sd", Bm, coef)
    return v


def tgkb_hat(Ah: np.ndarray, bh: np.ndarray, k: int):
    """k steps of Algorithm 4 on Fourier data.

    Returns W (n, m, k), Q (n, l, k+1), c (n, k), z (n, k+1): the real
    Fourier coefficients of the tubes c_i and z_i (Normalize makes them
    non-negative reals per slice), i.e. the per-slice bidiagonal entries.
    """
    AhH = _ct(Ah)
    q, z1 = normalize_hat(bh)
    Q, W, c, z = [q], [], [], [z1]
    w_prev = None
    for i in range(k):
        w = np.einsum("sij,sj->si", AhH, Q[i])
        if w_prev is not None:
            w = w - w_prev * z[i][:, None]
        w = _reorth(w, W)
        w, ci = normalize_hat(w)
        W.append(w)
        c.append(ci)
        qn = np.einsum("sij,sj->si", Ah, w) - Q[i] * ci[:, None]
        qn = _reorth(qn, Q)
        qn, zn = normalize_hat(qn)
        Q.append(qn)
        z.append(zn)
        w_prev = w
    return dict(W=np.stack(W, axis=2) if W else np.zeros(Ah.shape[:1] + (Ah.shape[2], 0), complex),
                Q=np.stack(Q, axis=2), c=np.stack(c, axis=1) if c else np.zeros((Ah.shape[0], 0)),
                z=np.stack(z, axis=1))


def bidiag(c_s: np.ndarray, z_s: np.ndarray, k: int) -> np.ndarray:
    """Lower bidiagonal P_k ((k+1) x k) of one slice: c on the diagonal,
    z_2..z_{k+1} below it (Section 4.3)."""
    P = np.zeros((k + 1, k))
    for i in range(k):
        P[i, i] = c_s[i]
        P[i + 1, i] = z_s[i + 1]
    return P


def _projected_ls(c, z, k):
    """Per slice: min ||P_k y - z_1 e_1|| by least squares (Algorithm 5).

    Returns y (n, k) and the per-slice residual norms (n,)."""
    n = c.shape[0]
    y = np.zeros((n, k))
    phi = np.zeros(n)
    for s in range(n):
        P = bidiag(c[s], z[s], k)
        rhs = np.zeros(k + 1)
        rhs[0] = z[s, 0]
        ys, *_ = np.linalg.lstsq(P, rhs, rcond=None)
        y[s] = ys
        phi[s] = np.linalg.norm(P @ ys - rhs)
    return y, phi


def tgkb_solve(A, B, delta, tau, k_max, k_fixed=None):
    n, l, m = A.shape
    k_max = min(k_max, min(l, m))
    if k_fixed is not None:
        k_max = k_fixed
    Ah, Bh = fft3(A), fft3(B)
    g = tgkb_hat(Ah, Bh[:, :, 0], k_max)
    td = tau * delta
    res = {}
    k, status = k_max, STATUS_NOT_CONVERGED
    for i in range(1, k_max + 1):
        _, phi = _projected_ls(g["c"], g["z"], i)
        res[i] = float(np.sqrt(np.sum(phi ** 2) / n))
        if res[i] <= td and k_fixed is None:
            k, status = i, STATUS_OK
            break
    if k_fixed is not None:
        status = STATUS_OK
    y, _ = _projected_ls(g["c"], g["z"], k)
    Xh = np.einsum("sdj,sj->sd", g["W"][:, :, :k], y)[:, :, None]
    return dict(X=ifft3_real(Xh), k=k, status=status, res=res, tau_delta=td,
                margin=_margin(res, k, td), W=g["W"][:, :, :k], Q=g["Q"][:, :, :k + 1],
                c=g["c"][:, :k], z=g["z"][:, :k + 1])


def ritz_triplets(A, B, k):
    """The analogues of Ritz triplets from k steps of Algorithm 4 (Section 4.3,
    Eq. (16)-(solgkbb)): per Fourier slice the SVD P_k = U_P S V_P^T of the
    (k+1) x k lower bidiagonal, and the triplets (s_i, Q_{k+1} U_P e_i,
    W_k V_P e_i), largest first.  Returns the Fourier factors Uh (n, l, k),
    S (n, k), Vh (n, m, k) and the spatial tensors U (n, l, k), s (n, k)
    tubes, V (n, m, k)."""
    Ah, Bh = fft3(A), fft3(B)
    g = tgkb_hat(Ah, Bh[:, :, 0], k)
    n = A.shape[0]
    Uh = np.zeros((n, A.shape[1], k), dtype=complex)
    Vh = np.zeros((n, A.shape[2], k), dtype=complex)
    S = np.zeros((n, k))
    for s in range(n):
        Us, ss, Vts = np.linalg.svd(bidiag(g["c"][s], g["z"][s], k), full_matrices=False)
        S[s] = ss
        Uh[s] = g["Q"][s][:, :k + 1] @ Us
        Vh[s] = g["W"][s][:, :k] @ Vts.T
    return dict(Uh=Uh, S=S, Vh=Vh, U=ifft3_real(Uh), s=ifft3_real(S[:, None, :])[:, 0, :], V=ifft3_real(Vh), gkb=g)


def tgkb_p_solve(A, B, deltas, tau, k_max):
    """tGKB_p (Section 1 and Section 4.3): problem (I6) with p lateral slices
    B_j, each with its own noise bound ||E_j||_F <= delta_j, solved by
    applying the tGKB method to every slice separately; slice j gets its own
    number of steps k_j.  Returns X (n, m, p) and the per-slice records."""
    n, l, p = B.shape
    deltas = np.broadcast_to(np.asarray(deltas, dtype=np.float64), (p,))
    outs = [tgkb_solve(A, B[:, :, j:j + 1], float(deltas[j]), tau, k_max) for j in range(p)]
    X = np.concatenate([o["X"] for o in outs], axis=2)
    return dict(X=X, k=[o["k"] for o in outs], status=[o["status"] for o in outs], per_slice=outs)


def nested_tgkb_p_solve(A, B, deltas, eta, k_max, k_init=2):
    """nested_tGKB_p (Algorithm 6): one t-Krylov basis, grown by Algorithm 4
    from the first lateral slice B_1, serves all p slices in turn.  For slice
    j the projected problem min ||P_k Y - Q_{k+1}^T * B_j||_F is solved in the
    current basis; while its residual is >= eta delta_j the basis is extended
    by one more step (k <- k + 1: the subspaces are nested, so "go to step 2"
    continues the same process rather than restarting it), and slice j + 1
    starts from the k that slice j ended with.  The first test is made at
    k = k_init.  k stops at k_max (status NOT_CONVERGED for a slice still
    above its bound there).  The residual tested is the projected one, as
    printed; the part of B_j outside the span of Q_{k+1} is not in it."""
    n, l, p = B.shape
    m = A.shape[2]
    k_max = min(k_max, min(l, m))
    deltas = np.broadcast_to(np.asarray(deltas, dtype=np.float64), (p,))
    Ah, Bh = fft3(A), fft3(B)
    g = tgkb_hat(Ah, Bh[:, :, 0], k_max)       # the process to k_max; its first k steps are the k-step process
    k = min(k_init, k_max)
    X = np.zeros((n, m, p), dtype=complex)
    ks, status, res_all = [], [], []
    for j in range(p):
        res = {}
        while True:
            Qk = g["Q"][:, :, :k + 1]
            rhs = np.einsum("sdi,sd->si", np.conj(Qk), Bh[:, :, j])     # Q_{k+1}^H b_j per slice
            y = np.zeros((n, k), dtype=complex)
            r2 = 0.0
            for s in range(n):
                P = bidiag(g["c"][s], g["z"][s], k)
                ys, *_ = np.linalg.lstsq(P, rhs[s], rcond=None)
                y[s] = ys
                r2 += float(np.sum(np.abs(P @ ys - rhs[s]) ** 2))
            res[k] = float(np.sqrt(r2 / n))
            if res[k] < eta * deltas[j]:
                st = STATUS_OK
                break
            if k >= k_max:
                st = STATUS_NOT_CONVERGED
                break
            k += 1
        X[:, :, j] = np.einsum("sdi,si->sd", g["W"][:, :, :k], y)
        ks.append(k)
        status.append(st)
        res_all.append(res)
    return dict(X=ifft3_real(X), k=ks, status=status, res=res_all, W=g["W"], Q=g["Q"])


# --------------------------------------------------------------------------
# tGKT: Tikhonov regularisation of the tGKB-projected problem (Section 5).
# --------------------------------------------------------------------------

def tikhonov_residual(U1: np.ndarray, S: np.ndarray, z1: np.ndarray, mu: float, n: int) -> float:
    """||P y_mu - z1 e1|| summed over slices (Parseval), from each slice's
    thin SVD P = U S V^T: sum_j (z1 u_1j / (1 + mu s_j^2))^2 + z1^2 (1 - sum_j u_1j^2)."""
    tot = 0.0
    for s in range(U1.shape[0]):
        f = z1[s] * U1[s] / (1.0 + mu * S[s] ** 2)
        tot += np.sum(f ** 2) + z1[s] ** 2 * max(1.0 - np.sum(U1[s] ** 2), 0.0)
    return float(np.sqrt(tot / n))


def _bidiag_svds(c, z, k):
    n = c.shape[0]
    U1 = np.zeros((n, k))
    S = np.zeros((n, k))
    Vs = np.zeros((n, k, k))
    for s in range(n):
        U, sv, VT = np.linalg.svd(bidiag(c[s], z[s], k), full_matrices=False)
        U1[s], S[s], Vs[s] = U[0], sv, VT.T
    return U1, S, Vs


def tikhonov_fixed_mu(g, mu):
    """Projected Tikhonov solution X = W_k * Y_mu for a given mu, from the
    output g of tgkb_solve (or of tgkb_hat plus k)."""
    n = g["c"].shape[0]
    k = g["c"].shape[1]
    U1, S, Vs = _bidiag_svds(g["c"], g["z"], k)
    z1 = g["z"][:, 0]
    y = np.zeros((n, k))
    for s in range(n):
        y[s] = Vs[s] @ (S[s] / (S[s] ** 2 + 1.0 / mu) * z1[s] * U1[s])
    Xh = np.einsum("sdj,sj->sd", g["W"], y)[:, :, None]
    return ifft3_real(Xh), tikhonov_residual(U1, S, z1, mu, n)


def tgkt_solve(A, B, delta, tau, k_max, mu_lo, mu_hi, log_tol=1e-12, max_iter=200):
    n, l, m = A.shape
    g = tgkb_solve(A, B, delta, tau, k_max)
    k = g["k"]
    c, z = g["c"], g["z"]
    U1, S, Vs = _bidiag_svds(c, z, k)
    z1 = z[:, 0]
    td = tau * delta
    lo, hi = np.log10(mu_lo), np.log10(mu_hi)
    status = STATUS_OK
    f = lambda t: tikhonov_residual(U1, S, z1, 10.0 ** t, n) - td
    if f(hi) > 0.0:
        t, status = hi, STATUS_NOT_CONVERGED
    elif f(lo) <= 0.0:
        t = lo
    else:
        it = 0
        while hi - lo > log_tol and it < max_iter:
            mid = 0.5 * (lo + hi)
            if f(mid) > 0.0:
                lo = mid
            else:
                hi = mid
            it += 1
        t = hi
    mu = 10.0 ** t
    y = np.zeros((n, k))
    for s in range(n):
        y[s] = Vs[s] @ (S[s] / (S[s] ** 2 + 1.0 / mu) * z1[s] * U1[s])
    Xh = np.einsum("sdj,sj->sd", g["W"], y)[:, :, None]
    return dict(X=ifft3_real(Xh), k=k, mu=mu, status=status, tau_delta=td,
                residual=tikhonov_residual(U1, S, z1, mu, n), gkb=g)


# --------------------------------------------------------------------------
# Gradients with respect to the tube weights of a separable operator.
# --------------------------------------------------------------------------

def tikhonov_rho(g, mu, G):
    """rho_s = <G-hat_s, dX-hat_s/d lam> (lam = 1/mu) for the projected
    Tikhonov solution of tikhonov_fixed_mu with the same g and mu: per slice
    y = V diag(S / (S^2 + lam)) U1 z1 from the SVD of the bidiagonal P_k, so
    dy/dlam = -V diag(S / (S^2 + lam)^2) U1 z1 and dX-hat/dlam = W_k dy/dlam.
    Returns the n complex values (full spectrum)."""
    n = g["c"].shape[0]
    k = g["c"].shape[1]
    U1, S, Vs = _bidiag_svds(g["c"], g["z"], k)
    z1 = g["z"][:, 0]
    lam = 1.0 / mu
    Gh = fft3(G)[:, :, 0]
    rho = np.zeros(n, complex)
    for s in range(n):
        dy = Vs[s] @ (-S[s] / (S[s] ** 2 + lam) ** 2 * z1[s] * U1[s])
        xi = g["W"][s] @ dy
        rho[s] = np.vdot(Gh[s], xi)
    return rho


def grad_c_separable(X, G, c, lam=0.0, rho=None):
    """dL/dc for a solution X (n, m, p) of a solve with the separable operator
    A(:,:,k) = c_k T, for G = dL/dX, with the discrete choices of the solve (k,
    the sketch rank r) held fixed.

    Each Fourier slice of A is c-hat_s T, and the subspaces every method builds
    from a slice (the RT-tSVD sketch with its power iterations, the tGKB
    Krylov space, the singular vectors) are those of T, so the truncated
    solutions are X-hat_s = M_s B-hat_s / c-hat_s with M_s free of c:
    dX-hat_s = -X-hat_s dc-hat_s / c-hat_s.  The projected Tikhonov solution
    with damping lam is z(lam / |c-hat_s|^2) / c-hat_s, z the solution for T,
    which adds -(2 lam / |c-hat_s|^2) xi_s Re(conj(c-hat_s) dc-hat_s) with
    xi_s = dX-hat_s/dlam (rho_s = <G-hat_s, xi_s> from tikhonov_rho).  With
    dL = (1/n) sum_s Re<G-hat_s, dX-hat_s> (Parseval) and dc-hat_s =
    sum_k dc_k w^{sk}, w = exp(-2 pi i / n):
        dL/dc_k = -(1/n) sum_s Re( (gamma_s + 2 lam Re rho_s) / c-hat_s * w^{sk} ),
    gamma_s = <G-hat_s, X-hat_s>.  The paper has no counterpart; the sum over
    s is written out over the full spectrum."""
    n = c.shape[0]
    Xh, Gh = fft3(X), fft3(G)
    ch = fft3(np.asarray(c, float)[:, None, None])[:, 0, 0]
    gam = np.einsum("sij,sij->s", np.conj(Gh), Xh)
    if rho is not None:
        gam = gam + 2.0 * lam * np.real(rho)
    a = -gam / ch
    idx = np.arange(n)
    w = np.exp(-2j * np.pi * np.outer(idx, idx) / n)
    return np.real(a @ w) / n


# --------------------------------------------------------------------------
# Gradient with respect to B of the Tikhonov-tGKB solution (Section 5) at a
# fixed number of steps k and a fixed mu.
# --------------------------------------------------------------------------

def tgkt_fixed(A, B, k, mu):
    """The Tikhonov-tGKB solution for one lateral slice B after k steps of
    Algorithm 4, at the given mu (no discrepancy choice of k or mu)."""
    g = tgkb_solve(A, B, 0.0, 1.0, k, k_fixed=k)
    X, _ = tikhonov_fixed_mu(g, mu)
    return X


def _gkb_slice_taped(a: np.ndarray, b: np.ndarray, k: int) -> dict:
    """k steps of Algorithm 4 on one Fourier slice (a: l x m, b: l) with the
    intermediate vectors kept for the reverse sweep; reorthogonalisation by
    two classical Gram-Schmidt passes, as tgkb_hat."""
    l, m = a.shape
    U = np.zeros((l, k + 1), complex)
    V = np.zeros((m, k), complex)
    al = np.zeros(k)
    be = np.zeros(k + 1)
    tape = []
    be[0] = np.linalg.norm(b)
    U[:, 0] = b / be[0]
    for j in range(k):
        w0 = a.conj().T @ U[:, j]
        if j > 0:
            w0 = w0 - be[j] * V[:, j - 1]
        w1 = w0 - V[:, :j] @ (V[:, :j].conj().T @ w0)
        w2 = w1 - V[:, :j] @ (V[:, :j].conj().T @ w1)
        al[j] = np.linalg.norm(w2)
        V[:, j] = w2 / al[j]
        t0 = a @ V[:, j] - al[j] * U[:, j]
        t1 = t0 - U[:, :j + 1] @ (U[:, :j + 1].conj().T @ t0)
        t2 = t1 - U[:, :j + 1] @ (U[:, :j + 1].conj().T @ t1)
        be[j + 1] = np.linalg.norm(t2)
        U[:, j + 1] = t2 / be[j + 1]
        tape.append((w0, w1, t0, t1))
    return dict(U=U, V=V, al=al, be=be, tape=tape)


def _unproject_bar(fbar: np.ndarray, x_in: np.ndarray, Q: np.ndarray, Qbar: np.ndarray) -> np.ndarray:
    """Reverse of f = x - Q (Q^H x) for a real loss: returns x-bar and adds
    the contribution to Q-bar (in place).  Bars follow dL = Re<bar, d.>."""
    if Q.shape[1] == 0:
        return fbar
    c = Q.conj().T @ x_in
    qf = Q.conj().T @ fbar
    Qbar -= np.outer(fbar, c.conj()) + np.outer(x_in, qf.conj())
    return fbar - Q @ qf


def _unnormalize_bar(ubar: np.ndarray, nbar: float, u: np.ndarray, nrm: float) -> np.ndarray:
    """Reverse of (u, nrm) = (t / ||t||, ||t||): t-bar from u-bar and nrm-bar."""
    return ubar / nrm + (nbar - np.real(np.vdot(u, ubar)) / nrm) * u


def tgkt_adjoint(A, B, k, mu, G):
    """dL/dB for L with dL/dX = G, X = tgkt_fixed(A, B, k, mu): the reverse
    (adjoint) sweep through the k steps of Algorithm 4 per Fourier slice, the
    reorthogonalisation and normalisations included, and through the
    projected Tikhonov solve y = (P_k^T P_k + I/mu)^{-1} P_k^T z_1 e_1.
    Returns (dB, X), both (n, l, 1) and (n, m, 1) real."""
    n, l, m = A.shape
    lam = 1.0 / mu
    Ah, Bh, Gh = fft3(A), fft3(B)[:, :, 0], fft3(G)[:, :, 0]
    Xh = np.zeros((n, m), complex)
    Yh = np.zeros((n, l), complex)
    for s in range(n):
        a = Ah[s]
        f = _gkb_slice_taped(a, Bh[s], k)
        U, V, al, be = f["U"], f["V"], f["al"], f["be"]
        P = bidiag(al, be, k)
        M = P.T @ P + lam * np.eye(k)
        y = np.linalg.solve(M, P.T @ (be[0] * np.eye(k + 1)[:, 0]))
        Xh[s] = V @ y
        # x = V y;  y = M^{-1} P^T be_0 e_1
        xbar = Gh[s]
        Vbar = np.outer(xbar, y)
        ybar = np.real(V.conj().T @ xbar)
        sv = np.linalg.solve(M, ybar)
        Pbar = np.outer(be[0] * np.eye(k + 1)[:, 0], sv) - P @ (np.outer(sv, y) + np.outer(y, sv))
        albar = np.array([Pbar[j, j] for j in range(k)])
        bebar = np.zeros(k + 1)
        bebar[0] = sv @ (P.T @ np.eye(k + 1)[:, 0])
        for j in range(k):
            bebar[j + 1] += Pbar[j + 1, j]
        Ubar = np.zeros_like(U)
        for j in range(k - 1, -1, -1):
            w0, w1, t0, t1 = f["tape"][j]
            t2bar = _unnormalize_bar(Ubar[:, j + 1], bebar[j + 1], U[:, j + 1], be[j + 1])
            Uj = U[:, :j + 1]
            Ujbar = np.zeros_like(Uj)
            t1bar = _unproject_bar(t2bar, t1, Uj, Ujbar)
            t0bar = _unproject_bar(t1bar, t0, Uj, Ujbar)
            Ubar[:, :j + 1] += Ujbar
            # t0 = a v_j - al_j u_j
            Vbar[:, j] += a.conj().T @ t0bar
            albar[j] -= np.real(np.vdot(U[:, j], t0bar))
            Ubar[:, j] -= al[j] * t0bar
            w2bar = _unnormalize_bar(Vbar[:, j], albar[j], V[:, j], al[j])
            Vj = V[:, :j]
            Vjbar = np.zeros_like(Vj)
            w1bar = _unproject_bar(w2bar, w1, Vj, Vjbar)
            w0bar = _unproject_bar(w1bar, w0, Vj, Vjbar)
            Vbar[:, :j] += Vjbar
            # w0 = a^H u_j - be_j v_{j-1}
            Ubar[:, j] += a @ w0bar
            if j > 0:
                bebar[j] -= np.real(np.vdot(V[:, j - 1], w0bar))
                Vbar[:, j - 1] -= be[j] * w0bar
        Yh[s] = _unnormalize_bar(Ubar[:, 0], bebar[0], U[:, 0], be[0])
    # dL = (1/n) sum_s Re<Gh_s, dXh_s> = (1/n) sum_s Re<Yh_s, dBh_s>, so dL/dB = Re(ifft(Yh))
    return ifft3_real(Yh[:, :, None]), ifft3_real(Xh[:, :, None])


# --------------------------------------------------------------------------
# t-Lanczos (Algorithm t-Lanc) and the t-Lanczos method (Eq. (9t)); symmetric A.
# --------------------------------------------------------------------------

def tlanczos_hat(Ah: np.ndarray, bh: np.ndarray, k: int):
    """k steps of the symmetric t-Lanczos process with reorthogonalisation."""
    q, z0 = normalize_hat(bh)
    Q, c, z = [q], [], []
    for i in range(k):
        v = np.einsum("sij,sj->si", Ah, Q[i])
        ci = np.einsum("si,si->s", np.conj(Q[i]), v)
        v = v - Q[i] * ci[:, None]
        if i > 0:
            v = v - Q[i - 1] * z[i - 1][:, None]
        v = _reorth(v, Q)
        v, zi = normalize_hat(v)
        Q.append(v)
        c.append(ci)
        z.append(zi)
    return dict(Q=np.stack(Q, axis=2), c=np.stack(c, axis=1), z=np.stack(z, axis=1), z0=z0)


def tridiag(c_s, z_s, k):
    """T_k ((k+1) x k): c on the diagonal, z on both off-diagonals."""
    T = np.zeros((k + 1, k), dtype=np.complex128)
    for i in range(k):
        T[i, i] = c_s[i]
        T[i + 1, i] = z_s[i]
        if i + 1 < k:
            T[i, i + 1] = z_s[i]
    return T


def tlanczos_solve(A, B, delta, tau, k_max):
    n, l, m = A.shape
    k_max = min(k_max, m)
    Ah, Bh = fft3(A), fft3(B)
    g = tlanczos_hat(Ah, Bh[:, :, 0], k_max)
    td = tau * delta
    res, ys = {}, {}
    k, status = k_max, STATUS_NOT_CONVERGED
    for i in range(1, k_max + 1):
        y = np.zeros((n, i), complex)
        tot = 0.0
        for s in range(n):
            T = tridiag(g["c"][s], g["z"][s], i)
            rhs = np.zeros(i + 1, complex)
            rhs[0] = g["z0"][s]
            y[s], *_ = np.linalg.lstsq(T, rhs, rcond=None)
            tot += np.linalg.norm(T @ y[s] - rhs) ** 2
        res[i] = float(np.sqrt(tot / n))
        ys[i] = y
        if res[i] <= td:
            k, status = i, STATUS_OK
            break
    Xh = np.einsum("sdj,sj->sd", g["Q"][:, :, :k], ys[k])[:, :, None]
    return dict(X=ifft3_real(Xh), k=k, status=status, res=res, tau_delta=td)
