// Host-side launchers shared between the translation units of libtprod.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "tprod.h"

namespace tp {

extern int g_launches;  // kernels enqueued by the library (reported by tp_kernel_launches)

inline tp_status cuda_status(cudaError_t e) { return e == cudaSuccess ? TP_OK : TP_ERR_CUDA; }

// Optional per-kernel-class device timing (tp_timing_enable / tp_timing_read):
// prof_begin records a start event before a launch of an enabled class and
// launched() records the matching end event.
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st);
// Opt a kernel into `bytes` of dynamic shared memory.  Always needed when
// static + dynamic shared memory exceeds 48 KB; cached per kernel.
tp_status smem_optin(const void* kern, size_t bytes);
// Bound of the waits for progress (grid-wide waits of the persistent tGKB
// kernels, mbarrier waits of the tensor-core product), in SM clock cycles:
// `dflt` unless tp_wait_budget set another.  Drains of work already in flight
// keep their own bound.
long long wait_budget(long long dflt);
// 1 when tp_wait_stall asked the grid-wide waits to wait for one arrival more
// than the grid makes (failure-detection tests), else 0.
int wait_stall();
// After a solve whose DFTs wrote norm partials of A and B: a NaN or infinity
// in either sum marks every one of the cnt info records TP_ERR_NONFINITE
// (residual NaN).  One small launch.
tp_status info_nonfinite(const double* partsA, int nA, const double* partsB, int nB, tp_info* info, int cnt,
                         cudaStream_t st);

inline tp_status launched(int cls, cudaStream_t st) {
    ++g_launches;
    prof_end(cls, st);
    return cuda_status(cudaGetLastError());
}

// Real <-> half-spectrum mode-3 DFT over a batch of tubes.  A "tube set" is
// rows x cols tubes; tube (r, c) of slice k sits at base + k*ss + r*ld + c.
// The spectrum is (h, rows, cols) contiguous.  sumsq (optional, device) gets
// one float64 partial sum of squares per CTA; nparts returns their count.
template <typename T>
tp_status rdft(const T* X, void* Xh, int n, int rows, int cols, long ld, long ss,
               double* sumsq, const int* skip, cudaStream_t st);
template <typename T>
tp_status irdft(const void* Xh, T* X, int n, int rows, int cols, long ld, long ss,
                const int* skip, cudaStream_t st);
int rdft_parts(int rows, int cols);
// ||X||_F^2 of the tensor whose half spectrum (n/2+1, rows, cols) is Xh, as the
// rdft_parts(rows, cols) partial sums that rdft writes for X (Parseval).
template <typename T>
tp_status norm2_hat(const void* Xh, int n, int rows, int cols, double* parts, cudaStream_t st);
size_t rdft_smem(int n, size_t elem);

// Batched complex matrix product over slices:
//   C[s] = alpha * op(A[s]) * op(B[s]) + beta * C[s]
// op bits: 1 = transpose, 2 = conjugate.  Row-major operands with leading
// dimensions and slice strides in complex elements.  dM/dN/dK (optional,
// device) cap the effective sizes at run time.  skip (optional, device):
// the launch does nothing when *skip != 0.
enum { OP_N = 0, OP_T = 1, OP_R = 2, OP_C = 3 };
// Float32 products with alpha = 1, beta = 0, op(B) = B, at most 32 columns,
// no run-time size caps and 16-byte aligned operands run on the tensor cores
// (zgemm_tc): tc_passes = 3 (3xTF32, float32 accuracy) or 1 (one tf32
// product, the TF32 precision form).  err (optional, device) receives
// TP_ERR_TIMEOUT if one of that kernel's bounded waits runs out.
template <typename T>
tp_status cgemm(int batch, int M, int N, int K, const int* dM, const int* dN, const int* dK,
                double alpha_re, double alpha_im, const void* A, long lda, long sA, int opA,
                const void* B, long ldb, long sB, int opB, double beta_re, double beta_im,
                void* C, long ldc, long sC, const int* skip, cudaStream_t st, int* err = nullptr,
                int tc_passes = 3);

// Tensor-core complex product C[s] = op(A[s]) B[s] (op = N, R or C), float32
// data, passes 3 or 1; TP_ERR_UNSUPPORTED (nothing enqueued) when the shape
// does not fit.  trans_out (op N / R): write C^T (C[c * ldc + row]).  ncap
// (optional, device) with c0: the launch does nothing when c0 >= *ncap (a
// column chunk past a run-time column count; B and C already offset by c0).
tp_status zgemm_tc(int batch, int M, int N, int K, const void* A, long lda, long sA, int opA, const void* B,
                   long ldb, long sB, void* C, long ldc, long sC, const int* skip, int* err, int passes,
                   cudaStream_t st, int trans_out = 0, const int* ncap = nullptr, int c0 = 0);

// The tensor-core product's stage-count tuner (a per-shape table consulted by
// every zgemm_tc launch; results do not depend on the stage count).
tp_status zgemm_tc_tune(int batch, int M, int N, int K, int opA, int passes, int trans_out, void* scratch,
                        size_t scratch_bytes, cudaStream_t st, int* ns_out, float* ms_out, float* ms_dflt);
int zgemm_tc_tuned(int* ints, float* flts, int max);
tp_status zgemm_tc_set(int op, int passes, int N, int M, int K, int batch, int ns);
void zgemm_tc_untune();

// Batched tGKB (tGKB_p): one cooperative launch carries GKM_PB lateral
// slices of B (columns j0 .. j0+pb-1) through Algorithm 4 in lockstep.
// Complex arrays are cplx<T>: Ahat (h, l, m), Bhat (h, l, p), Wb (h, PB,
// k_max, m), Qb (h, PB, k_max+1, l), Xhat (h, m, p); gv (h, PB, 3, k_max)
// Givens data; res2 (k_max+1, PB, h); counters (k_max+1, zeroed by the
// launcher); info: p records; res_hist (optional): (p, k_max+1).
constexpr int GKM_PB = 8;
struct GkmArgs {
    const void* Ahat;
    const void* Bhat;
    void* Wb;
    void* Qb;
    void* Xhat;
    double* gv;
    double* res2;
    unsigned* counters;
    tp_info* info;
    double* res_hist;
    long long spin;  // bound of each grid-wide wait, in SM clock cycles
    int extra;       // arrivals awaited beyond the grid (0; 1 under tp_wait_stall)
    int l, m, n, h, k_max, p, j0, pb;
    double td[GKM_PB];    // tau * delta_j
    double td2n[GKM_PB];  // n (tau delta_j)^2, compared with the Parseval sums
};
// Launch configuration of the batched kernel for these sizes (threads per
// CTA, dynamic shared memory); TP_ERR_UNSUPPORTED when its CTAs cannot all be
// resident or the rows of A are not 16-byte multiples.  Enqueues nothing.
template <typename T> tp_status gkm_config(int l, int m, int n, int k_max, int* nt, size_t* smem);
template <typename T> tp_status gkm_launch(const GkmArgs& a, int nt, size_t smem, cudaStream_t st);

// Device-side bookkeeping shared by a solve.
struct State {
    double norm_a2;   // ||A||_F^2
    double eps2;      // eps^2 of Algorithm 3
    double eta;       // error indicator
    double norm_b2;   // ||B||_F^2
    double sigma_max;
    int done;         // sketch finished
    int r;            // sketch rank reached
    int k;            // truncation index
    int status;
    int sweeps;
    int nonfinite;    // 1 when the norms of A or B are not finite
    unsigned arrived; // CTAs of the current block orthonormalisation that have finished (0 between launches)
    int pad;
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// One-sided Jacobi SVD of h square factors R (r x r complex, row-major, r =
// st->r <= r_max) per CTA, the np columns of d (r x np row-major) rotated
// along: sigma sorted decreasing, U_R (columns normalised) and d' = J^H d with
// rows in sorted order.  TP_ERR_UNSUPPORTED when the working set exceeds
// shared memory.
template <typename T>
tp_status jacobi_svd(int h, const void* R, long ldr, long sR, const State* st, const void* d, long sd, int np,
                     T* sigma, long ssig, void* UR, long ldu, long sU, void* dprime, long sdp, int r_max,
                     int* sweeps, cudaStream_t stream);

struct Carver {
    char* base;
    size_t off;
    size_t cap;
    explicit Carver(void* p, size_t c) : base((char*)p), off(0), cap(c) {}
    template <typename U> U* take(size_t count) {
        U* p = base ? (U*)(base + off) : nullptr;
        off = align256(off + count * sizeof(U));
        return p;
    }
};

// Gradients with respect to the tube weights of a separable operator
// (grad.cu).  sep_gamma: gamma[s] = <Gh[s], Xh[s]> over `per` complex entries
// per slice; grad_c: dc_k = -(1/n) sum_s Re((gamma_s + add_s) / c-hat_s w^{sk})
// over the half spectrum (add optional, device, h entries).
constexpr int GRAD_MAX_N = 1024;
template <typename T>
tp_status sep_gamma(const void* Xh, const void* Gh, int h, long per, double2* gamma, cudaStream_t st);
tp_status grad_c(const double* c, int n, const double2* gamma, const double* add, double* dc, cudaStream_t st);
template <typename T> size_t sep_ws_bytes(int m, int n, int p);
template <typename T>
tp_status sep_grad(const T* X, const T* G, const double* c, int m, int n, int p, double* dc, void* ws,
                   size_t ws_bytes, cudaStream_t st);
template <typename T>
tp_status sep_operator(const T* Tm, const double* c, int l, int m, int n, T* A, cudaStream_t st);
// dL/dB of the Tikhonov-tGKB solution left in solve_ws (k and mu held): the
// reverse sweep through Algorithm 4, one CTA per slice.  Ahat: null, or the
// caller's half spectrum when the solve was given one.
// The same for the solution of a single-slice tGKB solve (lam = 0).
template <typename T> size_t gk_adj_ws_bytes(int l, int m, int n, const tp_tgkb_params* P);
template <typename T>
tp_status gk_adjoint(const T* G, int l, int m, int n, const tp_tgkb_params* P, const void* solve_ws,
                     size_t solve_ws_bytes, const void* Ahat, T* dB, void* ws, size_t ws_bytes, cudaStream_t st);
template <typename T> size_t tik_adj_ws_bytes(int l, int m, int n, const tp_tik_params* P);
template <typename T>
tp_status tik_adjoint(const T* G, int l, int m, int n, const tp_tik_params* P, const void* solve_ws,
                      size_t solve_ws_bytes, const void* Ahat, T* dB, void* ws, size_t ws_bytes, cudaStream_t st);
template <typename T> size_t tik_grad_ws_bytes(int l, int m, int n, const tp_tik_params* P);
template <typename T>
tp_status tik_grad_c(const T* G, const double* c, int l, int m, int n, const tp_tik_params* P, const void* solve_ws,
                     size_t solve_ws_bytes, double* dc, void* ws, size_t ws_bytes, cudaStream_t st);

}  // namespace tp
