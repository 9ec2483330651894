/*
 * tprod.h -- C ABI of the GB300 t-product regularization library (libtprod.so).
 *
 * Operations follow Ugwu & Reichel, "Tensor regularization by truncated
 * iteration ... with a t-product" (arXiv 2110.02485):
 *   - the t-product and its mode-3 DFT (Section 2, Definition 2.1),
 *   - the RT-tSVD method (Algorithm 3, Section 4.2, Eq. (kinit)),
 *   - the tGKB method (Algorithm 4, Eqs. (t-gkb), (9tt), (solgkb)),
 *   - Tikhonov regularisation of the tGKB-projected problem (tGKT, Section 5),
 *   - the T-tSVD method (Section 4.1), tGKB_p and nested_tGKB_p (Algorithm 6),
 *     and the t-singular triplets of k tGKB steps (Section 4.3),
 * each with the discrepancy principle of Eq. (disp); and, with no counterpart
 * in the paper, gradients: the t-product's adjoint, dL/dB of the truncated
 * solutions, and dL/dc in the tube weights of a separable operator.
 *
 * Layouts (all row-major, all pointers DEVICE pointers owned by the caller):
 *   real tensor  l x m x n   : array (n, l, m); element (i,j,k) at [k*l*m + i*m + j]
 *   lateral slices l x p x n : array (n, l, p)
 *   Fourier tensor           : half spectrum, h = n/2 + 1 slices of l x m
 *                              complex values, interleaved (re, im), array (h, l, m)
 * The element type of every real/complex array is set by `prec`:
 *   TP_FP32 -> float / (float re, float im);  TP_FP64 -> double / (double, double).
 *
 * Streams: `stream` is a cudaStream_t passed as void*.  Every call only
 * enqueues work on that stream and returns; results are ready when the stream
 * reaches that point.  Solvers write their tp_info to DEVICE memory.
 *
 * Errors: argument and launch errors are returned synchronously (nothing is
 * enqueued on an argument error).  Algorithmic outcomes (discrepancy principle
 * not met within the caps, a wait that timed out) are written to
 * info->status; X then holds the last candidate solution.
 *
 * Memory: the library never allocates device memory on these paths.  Solvers
 * and tprod_gemm take a caller-provided workspace of at least the size that
 * the matching *_workspace_bytes() query returns; ws must be 256-byte aligned.
 */
#ifndef TPROD_H
#define TPROD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TP_OK = 0,
    TP_ERR_ARG = -1,            /* invalid argument (sizes, pointers, precision)      */
    TP_ERR_CUDA = -2,           /* a CUDA launch or attribute call failed              */
    TP_ERR_WORKSPACE = -3,      /* workspace missing, misaligned or too small          */
    TP_ERR_BREAKDOWN = -4,      /* reserved: exact breakdown reported by a solver      */
    TP_ERR_NOT_CONVERGED = -5,  /* discrepancy principle not met within r_max / k_max  */
    TP_ERR_TIMEOUT = -6,        /* a bounded device-side wait gave up                  */
    TP_ERR_UNSUPPORTED = -7,    /* valid request outside what this build supports      */
    TP_ERR_NONFINITE = -8       /* A or B holds a NaN or an infinity (from the norms    */
                                /* the DFTs form); the solution is then meaningless     */
} tp_status;

/* Arithmetic precision of a call.
 *   TP_FP32: float data; every product float32-accurate (the tensor-core
 *            products with at most 32 columns use the 3xTF32 split).
 *   TP_FP64: double data, double arithmetic (CUDA cores).
 *   TP_TF32: float data; the tensor-core products (tprod_gemm with at most 32
 *            columns, and the block sketch and power-iteration products of
 *            rtsvd_truncated_solve) take one tf32 product each (10-bit
 *            mantissa inputs, float32 accumulation) instead of the 3xTF32
 *            split; the re-projection B^H = A^H Y of each block and
 *            everything else stay as TP_FP32.  The reduced-precision form of
 *            the RT-tSVD sketch (Algorithm 3's products), accepted by
 *            tprod_gemm, rtsvd_truncated_solve and their workspace queries;
 *            any other entry point rejects it with TP_ERR_ARG (or returns 0).
 *   TP_BF16: float data; the block sketch and power-iteration products of
 *            rtsvd_truncated_solve[_hat] run on bfloat16 copies of A-hat and
 *            A-hat^T (made once per solve, in the workspace: its query with
 *            TP_BF16 counts them) and a bfloat16 right-hand side, as
 *            tensor-core products with float32 accumulation; the
 *            re-projection and everything else stay as TP_FP32.  Shapes the
 *            bfloat16 products do not take (l or m not a multiple of 4)
 *            return TP_ERR_ARG.  Accepted by the RT-tSVD entry points and
 *            their workspace query only. */
typedef enum { TP_FP32 = 0, TP_FP64 = 1, TP_TF32 = 2, TP_BF16 = 3 } tp_precision;

/* Result record of a solve, written to device memory. */
typedef struct {
    int status;         /* tp_status of the algorithm (TP_OK, TP_ERR_NOT_CONVERGED, ...)  */
    int k;              /* truncation index / number of tGKB steps chosen                 */
    int r;              /* RT-tSVD: sketch rank reached by Algorithm 3; tGKB: steps run   */
    int sweeps;         /* RT-tSVD: Jacobi sweeps used (max over slices); else bisection  */
    double residual;    /* ||B - A*X||_F of the returned X as the method measures it       */
    double tau_delta;   /* tau * delta                                                     */
    double eta;         /* RT-tSVD: final error indicator eta (Theorem 4.2); else unused  */
    double mu;          /* tGKT: regularisation parameter; else 0                          */
    double margin;      /* min over {k, k-1} of |res - tau*delta| / (tau*delta)            */
    double norm_a2;     /* ||A||_F^2                                                       */
} tp_info;

/* ---------------------------------------------------------------- DFT -----
 * tprod_fft: mode-3 DFT of a real tensor (Section 2: fft(A,[],3), the
 * unnormalised transform x_s = sum_k x_k exp(-2 pi i s k / n)), keeping the
 * h = n/2+1 non-redundant slices of the conjugate-symmetric result.
 *   A    : real (n, l, m)            Ahat : complex (h, l, m)
 * tprod_ifft: the inverse (with 1/n), reading a half spectrum and writing
 * the real tensor; the imaginary parts of slices 0 and n/2 are ignored.
 *   Xhat : complex (h, l, m)         X    : real (n, l, m)
 * Both: l, m, n >= 1.  No workspace.
 */
tp_status tprod_fft(const void* A, int l, int m, int n, void* Ahat, int prec, void* stream);
tp_status tprod_ifft(const void* Xhat, int l, int m, int n, void* X, int prec, void* stream);

/* ---------------------------------------------------------- t-product -----
 * tprod_gemm: C = op(A) * op(B), the t-product of Definition 2.1 computed as
 * mode-3 DFT, one complex matrix product per Fourier slice, inverse DFT.
 * op(X) = X^T is the t-transpose of Section 2 (each frontal slice transposed,
 * slices 2..n reversed), the adjoint of the t-product: for C = A * B,
 * dL/dA = G * B^T and dL/dB = A^T * G.  trans bit 0 selects op(A), bit 1
 * op(B):
 *   bit 0 clear: A is l x kk x n, array (n, l, kk);  set: A is kk x l x n, (n, kk, l)
 *   bit 1 clear: B is kk x m x n, array (n, kk, m);  set: B is m x kk x n, (n, m, kk)
 *   C : real (n, l, m)
 * Workspace: tprod_gemm_workspace_bytes(l, kk, m, n, prec).
 */
size_t tprod_gemm_workspace_bytes(int l, int kk, int m, int n, int prec);
tp_status tprod_gemm(const void* A, const void* B, void* C, int l, int kk, int m, int n,
                     int trans, int prec, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------- t-product, no allocation -----
 * tprod_gemm_noalloc: the same product as tprod_gemm, for callers that cannot
 * allocate device memory or pass a workspace (for example code inside a host
 * framework whose device memory belongs to an allocator it cannot reach, or a
 * latency-critical path that must not call cudaMalloc, which can block and
 * synchronise the device).  The paper has no counterpart: this is a service
 * of the library, not a step of the method.
 * The scratch is a static device array of 16 MiB inside the library, held by
 * every GPU that loads the library until the process exits.  A problem whose
 * three spectra need more than that returns TP_ERR_WORKSPACE and enqueues
 * nothing; the need is align256(h*l*kk*c) + align256(h*kk*m*c) +
 * align256(h*l*m*c) bytes, h = n/2+1, c = 8 (FP32) or 16 (FP64).  Sizes
 * that tprod_gemm refuses (an operand of 2^40 elements or more, l above
 * 65535*128) return TP_ERR_ARG, also before anything is enqueued.
 * The first call on each device looks up the array's device address (with
 * that device current); make it before any stream capture.  Calls share the
 * array, so calls that overlap on the GPU race; nothing needs clearing
 * between calls.  Arguments and layouts as tprod_gemm with trans bit 1
 * clear (transA = 0 or 1).
 */
tp_status tprod_gemm_noalloc(const void* A, const void* B, void* C, int l, int kk, int m, int n,
                             int transA, int prec, void* stream);

/* ----------------------------------------------------------- RT-tSVD ------
 * rtsvd_truncated_solve: the RT-tSVD method of Section 4.2.
 * Algorithm 3 in block form: Gaussian lateral slices are taken `block` at a
 * time from Omega (slice c of Omega is the c-th Gaussian slice G), sketched
 * with q_power power iterations, orthonormalised against the basis so far
 * (two classical Gram-Schmidt passes, then a Cholesky QR of the block, whose
 * basis equals the column-by-column Gram-Schmidt one up to rounding), and the
 * error indicator eta = ||A||_F^2 - ||Bt||_F^2 (Theorems 4.1-4.2) is updated
 * per block until eta < eps^2 or r = r_max.  The full tSVD of Bt gives
 * U_k = Q*U(:,1:k,:), S_k, V_k and X_k = V_k * S_k^{-1} * U_k^T * B; k is the
 * smallest index in [max(1, r - p_over), r] (Eq. (kinit)) with
 * ||B - A*X_k||_F <= tau*delta (Eq. (disp)), else k = r and status
 * TP_ERR_NOT_CONVERGED.  Singular values at or below max(l,m)*eps*sigma_max
 * are treated as zero.  With p > 1 lateral slices (problem (I6)) the slices
 * share the factorisation and one k, chosen from the Frobenius norm of the
 * residual over all slices (delta then bounds the norm of all of E).
 *   A     : real (n, l, m)       B : real (n, l, p)     X : real (n, m, p)
 *   Omega : real (n, m, r_max)   (Gaussian test slices, supplied by the caller)
 * Limits: 1 <= block <= 32; r_max <= min(l, m) and r_max <= 256; l, m <=
 * 1024; 1 <= p <= 64.  The small SVD keeps R's working copy in shared memory
 * while (r_max^2 + r_max p) complex entries fit in 227 KB, else in the
 * workspace (global memory, L2-resident); its r_max p right-hand sides must
 * fit in shared memory in either case; and the block orthonormalisation's
 * working set (about (l + 1) b + 2 r_max b complex entries) must fit too.
 * Float32 range: the small SVD forms squared inner products of the factor
 * (fourth powers of the data's magnitude), so float32 data far from unit
 * scale (entries of A near 1e-13, say) can end in TP_ERR_NOT_CONVERGED;
 * rescale such data, or use TP_FP64.
 */
typedef struct {
    double delta;       /* noise bound of Eq. (errbd)                                 */
    double tau;         /* discrepancy factor tau > 1                                 */
    double eps;         /* Algorithm 3 tolerance (absolute); if <= 0 use eps_rel      */
    double eps_rel;     /* tolerance relative to ||A||_F, used when eps <= 0          */
    int p_over;         /* oversampling rho of Eq. (kinit)                            */
    int q_power;        /* power iterations per block (0 = Algorithm 3's sketch)      */
    int block;          /* Gaussian slices per block (1 = Algorithm 3)                */
    int r_max;          /* cap on the sketch rank                                     */
    double* res_hist;   /* optional device array (r_max+1): ||B - A*X_k|| for
                           k in [k_init, r]; other entries set to -1                 */
} tp_rtsvd_params;

size_t rtsvd_workspace_bytes(int l, int m, int n, int p, const tp_rtsvd_params* params, int prec);
tp_status rtsvd_truncated_solve(const void* A, const void* B, const void* Omega,
                                int l, int m, int n, int p, const tp_rtsvd_params* params,
                                void* X, tp_info* d_info, int prec,
                                void* ws, size_t ws_bytes, void* stream);
/* rtsvd_truncated_solve_hat: the same solve from a precomputed half spectrum of A
 * (Section 2: every t-operation acts on the Fourier slices A-hat^(s)), so
 * that several solves with one operator transform it once (tprod_fft).
 * Ahat: device, (h = n/2+1, l, m) interleaved complex (complex64 for FP32 and
 * TF32, complex128 for FP64), 16-byte aligned, the layout tprod_fft writes;
 * read only, owned by the caller, and valid until the solve's work on the
 * stream is done.  Every other argument, the workspace size (the
 * *_workspace_bytes query) and the results are those of the plain call; the
 * solve forms ||A||_F^2 from A-hat by Parseval where it needs it (one
 * reduction over A-hat).  A null Ahat returns TP_ERR_ARG. */
tp_status rtsvd_truncated_solve_hat(const void* Ahat, const void* B, const void* Omega,
                                    int l, int m, int n, int p, const tp_rtsvd_params* params,
                                    void* X, tp_info* d_info, int prec,
                                    void* ws, size_t ws_bytes, void* stream);

/* rtsvd_adjoint: the adjoint of the map B -> X_k of the last
 * rtsvd_truncated_solve made with this workspace and the same arguments
 * (A, Omega, l, m, n, p, params, prec), for differentiation.  With k held at
 * the value that solve chose, X_k = V_k * S_k^{-1} * U_k^T * B is linear in
 * B, and for G = dL/dX_k
 *   dL/dB = U_k * S_k^{-1} * V_k^T * G,
 * the t-transpose of the filter (the adjoint of the t-product is the
 * t-transpose, Section 2).  It is formed from what the solve left in the
 * workspace: per Fourier slice U_k = Q Q^H K_k S_k^{-1} with K = A-hat V
 * (U-tilde_k = B-tilde V_k S_k^{-1}), so
 *   dB-hat = Q Q^H K_k S_k^{-2} V_k^H G-hat,
 * with the terms of singular values the solve treated as zero dropped.  The
 * paper has no counterpart; it is a service for gradient-based use.
 *   G : real (n, m, p)      dB : real (n, l, p)
 * The workspace must be untouched since that solve; the call overwrites the
 * solve's B-hat, d, alpha and X-hat scratch, not the factorisation, so it can
 * be repeated.  prec as for the solve (TP_TF32 computes as TP_FP32).
 */
tp_status rtsvd_adjoint(const void* G, int l, int m, int n, int p, const tp_rtsvd_params* params,
                        void* dB, int prec, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------ T-tSVD ------
 * ttsvd_solve: the T-tSVD method (Section 4.1, Eqs. (11)-(14)): the full tSVD
 * of A and X_s = sum_{i<=s} V_i * s_i^{-1} * U_i^T * B with the smallest s
 * whose residual ||B - A*X_s||_F <= tau*delta (Eq. (disp); else s = the last
 * index and TP_ERR_NOT_CONVERGED).  Computed by the RT-tSVD path with the
 * t-identity as the sketching tensor and r = min(l, m) (the sketch then spans
 * the whole range of A, and B-tilde has A's singular values), no power
 * iterations, the scan of Eq. (disp) from s = 1.  Singular values at or below
 * max(l,m)*eps*sigma_max are treated as zero.  B (n, l, p), X (n, m, p); p > 1
 * slices share one s (as rtsvd_truncated_solve).
 * Limits: min(l, m) <= 256, and as rtsvd_truncated_solve (with r_max = min(l, m)).
 */
typedef struct {
    double delta;       /* noise bound of Eq. (errbd)                                 */
    double tau;         /* discrepancy factor                                         */
    double* res_hist;   /* optional device array (min(l,m)+1): residual at each s    */
} tp_ttsvd_params;

size_t ttsvd_workspace_bytes(int l, int m, int n, int p, const tp_ttsvd_params* params, int prec);
tp_status ttsvd_solve(const void* A, const void* B, int l, int m, int n, int p,
                      const tp_ttsvd_params* params, void* X, tp_info* d_info, int prec,
                      void* ws, size_t ws_bytes, void* stream);

/* ttsvd_adjoint: the adjoint of the map B -> X_s of the last ttsvd_solve made
 * with this workspace and the same (l, m, n, p, params, prec).  With s held
 * at the value that solve chose, X_s is linear in B and for G = dL/dX_s
 *   dL/dB = U_s * S_s^{-1} * V_s^T * G
 * (as rtsvd_adjoint, on the factorisation the solve left in the workspace).
 *   G : real (n, m, p)      dB : real (n, l, p)
 * The workspace must be untouched since that solve; the call can be repeated.
 * The paper has no counterpart; it is a service for gradient-based use.
 */
tp_status ttsvd_adjoint(const void* G, int l, int m, int n, int p, const tp_ttsvd_params* params, void* dB, int prec,
                        void* ws, size_t ws_bytes, void* stream);

/* -------------------------------------------------------------- tGKB ------
 * tgkb_solve: the tGKB method (Algorithm 4 with both reorthogonalisation
 * steps done as two classical Gram-Schmidt passes).  After step i the
 * projected problem min ||P_i * Y - e_1 * z_1||_F (Eq. (9tt)) is solved per
 * Fourier slice (Givens QR of the lower-bidiagonal slice of P_i); the first i
 * with residual <= tau*delta gives k and X_k = W_k * Y_k (Eq. (solgkb)).
 * Normalize's breakdown branch (a zero Fourier slice) yields a zero vector
 * and a zero coefficient.  The whole iteration is one persistent launch with
 * one CTA per Fourier slice; its grid-wide wait is bounded (info->status
 * TP_ERR_TIMEOUT if it gives up).
 * With p > 1 lateral slices this is the tGKB_p method (Sections 1 and 4.3,
 * problem (I6) with ||E_j||_F <= delta_j): every slice B_j is solved on its
 * own, with its own bound delta_j and its own number of steps k_j.  Groups
 * of 8 slices go through the iteration together in one launch, sharing the
 * two products with A of each step; shapes that launch does not take (float
 * data with odd m, or too little shared memory) run one launch per slice.
 *   A : real (n, l, m)     B : real (n, l, p)     X : real (n, m, p)
 *   d_info : p device records, record j for slice j
 * Limits: k_max <= min(l, m, 512); l, m <= 1024; 1 <= p <= 1024; n <= 1024
 * (float32) or 512 (float64).  The persistent launch holds the CTAs of all
 * n/2 + 1 Fourier slices at once (one, two or four per SM: 1024, 512 or 256
 * threads each); a shape whose CTAs do not all fit returns
 * TP_ERR_UNSUPPORTED before anything is enqueued.
 */
typedef struct {
    double delta;       /* noise bound of Eq. (errbd); with p > 1, the bound of every
                           slice unless delta_p is given                               */
    double tau;         /* discrepancy factor                                         */
    int k_max;          /* step cap                                                   */
    double* res_hist;   /* optional device array, (k_max+1) entries per lateral slice
                           (slice-major): residual after step i, -1 where not formed   */
    const double* delta_p; /* optional HOST array of p bounds delta_j (p > 1); read
                              before the call returns                                  */
} tp_tgkb_params;

size_t tgkb_workspace_bytes(int l, int m, int n, int p, const tp_tgkb_params* params, int prec);
tp_status tgkb_solve(const void* A, const void* B, int l, int m, int n, int p,
                     const tp_tgkb_params* params, void* X, tp_info* d_info, int prec,
                     void* ws, size_t ws_bytes, void* stream);
/* tgkb_solve_hat: the same solve from a precomputed half spectrum of A
 * (Section 2: every t-operation acts on the Fourier slices A-hat^(s)), so
 * that several solves with one operator transform it once (tprod_fft).
 * Ahat: device, (h = n/2+1, l, m) interleaved complex (complex64 for FP32 and
 * TF32, complex128 for FP64), 16-byte aligned, the layout tprod_fft writes;
 * read only, owned by the caller, and valid until the solve's work on the
 * stream is done.  Every other argument, the workspace size (the
 * *_workspace_bytes query) and the results are those of the plain call; the
 * solve forms ||A||_F^2 from A-hat by Parseval where it needs it (one
 * reduction over A-hat).  A null Ahat returns TP_ERR_ARG. */
tp_status tgkb_solve_hat(const void* Ahat, const void* B, int l, int m, int n, int p,
                         const tp_tgkb_params* params, void* X, tp_info* d_info, int prec,
                         void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------ nested_tGKB_p ----
 * nested_tgkb_solve: the nested_tGKB_p method (Algorithm 6) for p lateral
 * slices.  One t-Krylov basis, grown by Algorithm 4 from B_1 (both
 * reorthogonalisations as in tgkb_solve), serves the slices in turn: slice j
 * solves its projected problem min ||P_k * Y - Q_{k+1}^T * B_j||_F in the
 * present basis; while that residual is >= tau * delta_j the basis is
 * extended by one step (the subspaces are nested: the same process goes on),
 * and slice j+1 starts from the k that slice j ended with.  The first test is
 * made at k = 2 (Algorithm 6's k_init).  The residual tested is the projected
 * one, as Algorithm 6 prints it.  params as for tgkb_solve (tau is Algorithm
 * 6's eta; delta_p optional); at k = k_max a slice above its bound is
 * accepted with TP_ERR_NOT_CONVERGED.  One persistent launch (one CTA per
 * Fourier slice, bounded grid-wide waits).
 *   A : real (n, l, m)     B : real (n, l, p)     X : real (n, m, p)
 *   d_info : p device records; res_hist (optional): (p, k_max+1), -1 where a
 *   slice was not tested.
 * Limits as tgkb_solve.
 */
size_t nested_tgkb_workspace_bytes(int l, int m, int n, int p, const tp_tgkb_params* params, int prec);
tp_status nested_tgkb_solve(const void* A, const void* B, int l, int m, int n, int p,
                            const tp_tgkb_params* params, void* X, tp_info* d_info, int prec,
                            void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------- tGKB t-singular triplets --
 * tgkb_triplets: the analogues of Ritz triplets of Section 4.3: k steps of
 * Algorithm 4 from B (no discrepancy stop), then per Fourier slice the SVD
 * P_k = U_P S V_P^T of the (k+1) x k lower bidiagonal, and the triplets
 * (s_i, Q_{k+1} * U_i, W_k * V_i), i = 1..k, largest first in every slice:
 * approximations of the k largest t-singular triplets of A, from which
 * Eq. (solgkbb) rebuilds the tGKB solution.
 *   A : real (n, l, m)   B : real (n, l, 1)
 *   U : real (n, l, k)   S : real (n, k), tube i in column i   V : real (n, m, k)
 * Limits as tgkb_solve, and (k+1)^2 complex entries twice in 227 KB of
 * shared memory (k <= 118 in FP32, 83 in FP64).
 */
size_t tgkb_triplets_workspace_bytes(int l, int m, int n, int k, int prec);
tp_status tgkb_triplets(const void* A, const void* B, int l, int m, int n, int k, void* U, void* S, void* V,
                        int prec, void* ws, size_t ws_bytes, void* stream);

/* -------------------------------------------------------------- tGKT ------
 * tgkb_tikhonov_solve: tGKB as above fixes k; then per Fourier slice
 *   y_mu = argmin ||P_k y - z_1 e_1||^2 + mu^{-1} ||y||^2
 * with one scalar mu for all slices, chosen on log10(mu) in [mu_lo, mu_hi]
 * (Section 5) so that ||B - A*X_mu||_F = tau*delta, to a bracket width of
 * log_tol in log10(mu).  If even mu_hi leaves the residual above tau*delta,
 * mu = mu_hi and status TP_ERR_NOT_CONVERGED; if mu_lo already meets it,
 * mu = mu_lo.  X = W_k * Y_mu.  One lateral slice (p = 1; gkb.delta_p is
 * ignored).
 */
typedef struct {
    tp_tgkb_params gkb;
    double mu_lo, mu_hi;   /* search interval, 0 < mu_lo < mu_hi                       */
    double log_tol;        /* bracket width in log10(mu); <= 0 selects 1e-12; float32
                              stops at 1e-7, the spacing of float32 mu^(-1/2)           */
} tp_tik_params;

size_t tgkb_tikhonov_workspace_bytes(int l, int m, int n, int p, const tp_tik_params* params, int prec);
tp_status tgkb_tikhonov_solve(const void* A, const void* B, int l, int m, int n, int p,
                              const tp_tik_params* params, void* X, tp_info* d_info, int prec,
                              void* ws, size_t ws_bytes, void* stream);
/* tgkb_tikhonov_solve_hat: the same solve from a precomputed half spectrum of A
 * (Section 2: every t-operation acts on the Fourier slices A-hat^(s)), so
 * that several solves with one operator transform it once (tprod_fft).
 * Ahat: device, (h = n/2+1, l, m) interleaved complex (complex64 for FP32 and
 * TF32, complex128 for FP64), 16-byte aligned, the layout tprod_fft writes;
 * read only, owned by the caller, and valid until the solve's work on the
 * stream is done.  Every other argument, the workspace size (the
 * *_workspace_bytes query) and the results are those of the plain call; the
 * solve forms ||A||_F^2 from A-hat by Parseval where it needs it (one
 * reduction over A-hat).  A null Ahat returns TP_ERR_ARG. */
tp_status tgkb_tikhonov_solve_hat(const void* Ahat, const void* B, int l, int m, int n, int p,
                                  const tp_tik_params* params, void* X, tp_info* d_info, int prec,
                                  void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------ gradients in the tube weights -------
 * For a separable operator A(:,:,k) = c_k T (one fixed l x m matrix T, tube
 * weights c: the blur law of the synthetic problems), every Fourier slice is
 * c-hat_s T (c-hat = fft(c)), and the subspaces the solvers build from a
 * slice (the RT-tSVD sketch with its power iterations for a fixed Omega, the
 * tGKB Krylov space, the singular vectors) are those of T.  With the discrete
 * choices of a solve held fixed (k, the sketch rank r, mu) its solution is
 * therefore X-hat_s = M_s B-hat_s / c-hat_s with M_s free of c for the
 * truncated methods, and z(lam / |c-hat_s|^2) / c-hat_s for the projected
 * Tikhonov solution with damping lam = 1/mu (z the solution for T).  For a
 * loss L with G = dL/dX, Parseval gives
 *   dL/dc_k = -(1/n) sum_{s<n} Re( (gamma_s + t_s) / c-hat_s * w^{sk} ),
 *   gamma_s = <G-hat_s, X-hat_s>,  w = exp(-2 pi i / n),
 * with t_s = 0 for the truncated methods and t_s = 2 lam Re<G-hat_s,
 * dX-hat_s/dlam> for the Tikhonov-tGKB solution.  A slice with c-hat_s = 0
 * contributes nothing.  The paper has no counterpart; these are services for
 * gradient-based use.  c and dc are float64 device arrays of n entries.
 * Limits: n <= 1024.
 *
 * sep_grad_c: for a solution X of rtsvd_truncated_solve, ttsvd_solve,
 * tgkb_solve or nested_tgkb_solve with such an operator.
 *   X, G : real (n, m, p);  m, p <= 4096.
 * Workspace: sep_grad_c_workspace_bytes(m, n, p, prec) (0: invalid sizes).
 */
/* sep_operator: forms the separable operator A(:,:,k) = c_k T on the device
 * (the product in float64, rounded once to the working precision), for
 * callers that differentiate in c.
 *   T : real (l, m)      c : device float64 (n)      A : real (n, l, m)
 * No workspace.
 */
tp_status sep_operator(const void* T, const double* c, int l, int m, int n, void* A, int prec, void* stream);

size_t sep_grad_c_workspace_bytes(int m, int n, int p, int prec);
tp_status sep_grad_c(const void* X, const void* G, const double* c, int m, int n, int p, double* dc, int prec,
                     void* ws, size_t ws_bytes, void* stream);

/* tgkb_tikhonov_grad_c: the same for the solution of the last
 * tgkb_tikhonov_solve made with solve_ws and the same (l, m, n, params,
 * prec), at the k and mu it chose, read from that workspace (untouched since;
 * this call does not modify it, so it can be repeated).  Per slice the
 * projected solution is y = M^{-1} P_k^T z_1 e_1 with M = P_k^T P_k + lam I,
 * so dX-hat/dlam = -W_k M^{-1} y, formed in float64 from the bidiagonal.
 *   G : real (n, m, 1)
 * Workspace: tgkb_tikhonov_grad_c_workspace_bytes(l, m, n, params, prec).
 */
size_t tgkb_tikhonov_grad_c_workspace_bytes(int l, int m, int n, const tp_tik_params* params, int prec);
tp_status tgkb_tikhonov_grad_c(const void* G, const double* c, int l, int m, int n, const tp_tik_params* params,
                               const void* solve_ws, size_t solve_ws_bytes, double* dc, int prec, void* ws,
                               size_t ws_bytes, void* stream);

/* --------------------------------- gradient of the Tikhonov-tGKB solution in B
 * tgkb_tikhonov_adjoint: dL/dB for a loss L of the solution X of the last
 * tgkb_tikhonov_solve (or _hat) made with solve_ws and the same (l, m, n,
 * params, prec), with the number of steps k and mu held at the values that
 * solve chose (Section 5: per Fourier slice the minimiser of ||A x - b||^2 +
 * mu^{-1} ||x||^2 over the Krylov space that k steps of Algorithm 4 build from
 * b).  The Krylov space moves with B and its motion is part of the gradient:
 * the call runs the reverse (adjoint) sweep through the k steps of Algorithm
 * 4 per slice, the two Gram-Schmidt passes and the Normalize steps included,
 * and through the projected Tikhonov solve, recomputing each step's vectors
 * from the two bases the solve kept (four products with A-hat per step; one
 * CTA per slice).  The paper has no counterpart; it is a service for
 * gradient-based use.
 *   G     : real (n, m, 1), dL/dX         dB : real (n, l, 1), written
 *   Ahat  : null when the solve transformed A itself; otherwise the same
 *           half spectrum (n/2+1, l, m) that was given to the _hat solve
 *           (read only, 16-byte aligned)
 * solve_ws is read, never modified (the call can be repeated).  Asynchronous
 * on the stream.  TP_ERR_ARG for null pointers or a misaligned Ahat;
 * TP_ERR_WORKSPACE when solve_ws or ws is too small or not 256-byte aligned.
 * Workspace: tgkb_tikhonov_adjoint_workspace_bytes(l, m, n, params, prec)
 * (0: invalid sizes).
 */
size_t tgkb_tikhonov_adjoint_workspace_bytes(int l, int m, int n, const tp_tik_params* params, int prec);
tp_status tgkb_tikhonov_adjoint(const void* G, int l, int m, int n, const tp_tik_params* params,
                                const void* solve_ws, size_t solve_ws_bytes, const void* Ahat, void* dB, int prec,
                                void* ws, size_t ws_bytes, void* stream);

/* tgkb_adjoint: the same for the solution of the last tgkb_solve (or _hat)
 * with one lateral slice (p = 1) made with solve_ws and the same (l, m, n,
 * params, prec), at the k it chose (Algorithm 4 and Eq. (solgkb): the least-
 * squares solution over the Krylov space, the Tikhonov case with mu^{-1} = 0).
 * Arguments, ownership and errors as tgkb_tikhonov_adjoint; a workspace of a
 * tGKB_p solve (p > 1) is laid out differently and must not be passed.
 * Workspace: tgkb_adjoint_workspace_bytes(l, m, n, params, prec).
 */
size_t tgkb_adjoint_workspace_bytes(int l, int m, int n, const tp_tgkb_params* params, int prec);
tp_status tgkb_adjoint(const void* G, int l, int m, int n, const tp_tgkb_params* params, const void* solve_ws,
                       size_t solve_ws_bytes, const void* Ahat, void* dB, int prec, void* ws, size_t ws_bytes,
                       void* stream);

/* --------------------------------------------------------- autotuner -------
 * rtsvd_autotune: picks, for every tensor-core product that an
 * rtsvd_truncated_solve with these sizes, params (block, r_max) and prec
 * launches, the stage count of the product's TMA ring (2 up to what one CTA's
 * shared memory holds; two CTAs per SM at two stages, one above) by timing
 * each candidate with CUDA events on scratch operands, and records the
 * fastest in a process-wide table that every later launch of that shape
 * consults.  Results do not depend on the stage count (the same MMAs in the
 * same order), only the time does.  The shapes: the sketch and power-iteration
 * products (A-hat Omega_b, A-hat Z; A-hat^H Y from the transposed copy) in the
 * sketch precision, the re-projection A-hat^H Y and the 32-column chunks of K
 * = A-hat V.  No counterpart in the paper.
 *   ws : device scratch, 256-byte aligned, at least rtsvd_workspace_bytes for
 *        the same arguments (its contents are overwritten)
 * Synchronises the stream (not for CUDA graph capture).  TP_FP64 tunes nothing
 * (the float64 products run on the SIMT kernel) and returns TP_OK.
 * TP_ERR_ARG for invalid sizes or precision; TP_ERR_WORKSPACE for a missing,
 * misaligned or too small ws.
 * tp_autotune_table: up to max entries of the table, entry i as ints[8 i ..
 *   8 i + 7] = (op: 0 A, 2 conj(A); passes: 3 float32-accurate, 1 tf32, 0
 *   bfloat16; columns rounded up to 8; M; K; batch; stages chosen; the
 *   built-in rule's stages) and flts[2 i .. 2 i + 1] = (ms of the choice, ms
 *   of the built-in rule); returns the number of entries written.
 * tp_autotune_clear: empties the table (every shape back to the built-in rule).
 * tp_autotune_set: puts one shape's stage count into the table (a stored
 *   tuning, or a test): op 0 (A), 2 (conj(A), from the transposed copy) or 3
 *   (A^H), passes, columns (1..32), M, K, batch as above; TP_ERR_ARG for a
 *   shape the tensor-core product does not take or a stage count outside 2 ..
 *   what fits.  Host only.
 */
tp_status rtsvd_autotune(int l, int m, int n, int p, const tp_rtsvd_params* params, int prec, void* ws,
                         size_t ws_bytes, void* stream);
int tp_autotune_table(int* ints, float* flts, int max);
void tp_autotune_clear(void);
tp_status tp_autotune_set(int op, int passes, int columns, int M, int K, int batch, int stages);

/* ------------------------------------------------------------ misc -------- */
const char* tp_status_string(int status);
int tp_version(void);                 /* 100 * major + minor                        */
int tp_kernel_launches(void);         /* kernels enqueued by this library so far    */
/* tp_wait_budget: the bound, in SM clock cycles, of every device-side wait for
 * progress in kernels launched after the call: the grid-wide waits of the
 * persistent tGKB kernels (Algorithm 4; default about 2 s) and the mbarrier
 * waits of the tensor-core product (default about 1 s).  0 restores the
 * defaults; a negative value returns TP_ERR_ARG.  A wait that runs out makes
 * its kernel stop its loop, drain the copies and tensor-core operations it
 * has in flight (those drains keep their own bound) and report TP_ERR_TIMEOUT
 * in the solve's tp_info; the context stays usable.  It exists for
 * failure-detection tests: a budget of a few cycles makes the waits run out
 * on purpose.  Process-wide; not meant to change while launches are being
 * enqueued from other threads. */
int tp_wait_budget(long long cycles);
/* tp_wait_stall: with on = 1, the grid-wide waits of the persistent tGKB
 * kernels launched after the call wait for one arrival more than their grid
 * makes, so that every such wait runs out after its budget (an arrival that
 * nothing makes); on = 0 restores normal waits.  For failure-detection tests
 * only, together with a short tp_wait_budget; the kernels then stop, report
 * TP_ERR_TIMEOUT and leave the context usable.  Process-wide. */
int tp_wait_stall(int on);

/* Optional device timing per kernel class, for benchmarks (off by default).
 * tp_timing_enable(mask): bit c of mask enables class c; every later launch
 * of an enabled class is bracketed by CUDA events on its stream (a few
 * microseconds of host time per launch).  mask = 0 disables.  Inside a
 * stream capture the events become external event-record nodes of the graph,
 * so each replay records them again.
 * tp_timing_read(ms, launches, nclasses): waits for the recorded events,
 * writes per class the summed device time (ms) and launch count (for
 * captured events: those of the latest replay), clears the record, and
 * returns the number of classes (TP_KC_COUNT) or a negative tp_status.  Not
 * for use while a stream is being captured; read once per capture (the
 * events go back to the library's pool). */
enum {
    TP_KC_DFT = 0,      /* mode-3 DFT / inverse DFT                               */
    TP_KC_GEMM = 1,     /* batched complex products over Fourier slices           */
    TP_KC_ORTH = 2,     /* block orthonormalisation (Algorithm 3 steps 5-9)       */
    TP_KC_SVD = 3,      /* one-sided Jacobi SVD of the projected factor           */
    TP_KC_GKB = 4,      /* persistent tGKB iteration (Algorithm 4)                */
    TP_KC_DP = 5,       /* discrepancy-principle scans and reductions             */
    TP_KC_TIK = 6,      /* Tikhonov parameter search and solution                 */
    TP_KC_MISC = 7,     /* small bookkeeping kernels                              */
    TP_KC_COUNT = 8
};
int tp_timing_enable(int class_mask);
int tp_timing_read(double* ms, int* launches, int nclasses);

#ifdef __cplusplus
}
#endif
#endif /* TPROD_H */
