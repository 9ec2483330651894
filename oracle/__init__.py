"""Plain FP64 CPU oracle for the t-product regularization methods.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
bench's CPU-baseline arm may import this package.  It shares no code with the
CUDA library; the only common module is the seeded input generator
(paper_2110_02485_gb300.synth), which holds no solver arithmetic.

Functions follow Ugwu & Reichel, "Tensor regularization by truncated
iteration: a comparison of some solution methods for large-scale linear
discrete ill-posed problem with a t-product" (arXiv 2110.02485): the
t-product algebra of Section 2 (talgebra) and the T-tSVD, RT-tSVD (Algorithm 3),
tGKB (Algorithm 4), Tikhonov-tGKB and t-Lanczos methods with the discrepancy
principle (methods).  The parity status of each function is recorded with its
pins in the test suite (tests/test_oracle_*.py); every function here is
pinned.
"""
from .talgebra import (fft3, ifft3, ifft3_real, dft3_naive, fro2, fro2_hat, tprod, bcirc,
                       unfold, fold, tprod_bcirc, ttranspose, tidentity, e1_tube,
                       normalize_hat, normalize, tube_norm, tsvd_hat, tsvd)
from .methods import (STATUS_OK, STATUS_NOT_CONVERGED, ttsvd_solve, ttsvd_adjoint, rtsvd_alg3, rtsvd_block, rtsvd_prefix,
                      rtsvd_solve, rtsvd_adjoint, tgkb_hat, tgkb_solve, tgkb_p_solve, ritz_triplets, nested_tgkb_p_solve, bidiag, tgkt_solve, tikhonov_fixed_mu,
                      tikhonov_residual, tlanczos_hat, tlanczos_solve, tridiag,
                      tikhonov_rho, grad_c_separable, tgkt_fixed, tgkt_adjoint)
