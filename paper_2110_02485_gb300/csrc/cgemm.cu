// Batched complex matrix product over Fourier slices (the facewise products
// of the t-product, Section 2): C[s] = alpha op(A[s]) op(B[s]) + beta C[s].
//
// Register-tiled SIMT kernel: a CTA computes a BM x BN tile of one slice,
// staging BK-deep slices of op(A) and op(B) in shared memory (double buffered
// through registers); each thread owns a TM x TN block of complex accumulators
// strided across the tile so that shared-memory reads are broadcasts or
// consecutive.  Operands are read with the contiguous dimension on
// consecutive threads whatever the op, so both A and A^H stream coalesced.
#include "common.cuh"
#include "internal.h"

namespace tp {

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_cgemm(int M, int N, int K, const int* dM, const int* dN, const int* dK, cplx<T> alpha,
        const cplx<T>* __restrict__ A, long lda, long sA, int opA, const cplx<T>* __restrict__ B, long ldb,
        long sB, int opB, cplx<T> beta, cplx<T>* __restrict__ C, long ldc, long sC, const int* skip) {
    typedef cplx<T> V;
    constexpr int TX = BN / TN, TY = BM / TM, NT = TX * TY;
    constexpr int AE = (BM * BK + NT - 1) / NT, BE = (BN * BK + NT - 1) / NT;
    constexpr int LDA_S = BM + 1, LDB_S = BN + 1;
    if (skip && *skip) return;
    int Me = M, Ne = N, Ke = K;
    if (dM) Me = min(Me, *dM);
    if (dN) Ne = min(Ne, *dN);
    if (dK) Ke = min(Ke, *dK);
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (m0 >= Me || n0 >= Ne) return;
    const long s = blockIdx.z;
    A += s * sA;
    B += s * sB;
    C += s * sC;

    extern __shared__ __align__(16) unsigned char smraw[];
    V* As = (V*)smraw;                    // [2][BK][LDA_S]
    V* Bs = As + 2 * BK * LDA_S;          // [2][BK][LDB_S]

    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const bool tA = opA & 1, cA = opA & 2, tB = opB & 1, cB = opB & 2;

    V ra[AE], rb[BE];
    auto loadA = [&](int k0) {
#pragma unroll
        for (int i = 0; i < AE; ++i) {
            const int e = tid + i * NT;
            V v = mk<T>(0, 0);
            if (e < BM * BK) {
                int mm, kk;
                if (tA) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
                const int gm = m0 + mm, gk = k0 + kk;
                if (gm < Me && gk < Ke) v = tA ? A[(long)gk * lda + gm] : A[(long)gm * lda + gk];
                if (cA) v.y = -v.y;
            }
            ra[i] = v;
        }
    };
    auto loadB = [&](int k0) {
#pragma unroll
        for (int i = 0; i < BE; ++i) {
            const int e = tid + i * NT;
            V v = mk<T>(0, 0);
            if (e < BN * BK) {
                int nn, kk;
                if (tB) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
                const int gn = n0 + nn, gk = k0 + kk;
                if (gn < Ne && gk < Ke) v = tB ? B[(long)gn * ldb + gk] : B[(long)gk * ldb + gn];
                if (cB) v.y = -v.y;
            }
            rb[i] = v;
        }
    };
    auto storeA = [&](int buf) {
#pragma unroll
        for (int i = 0; i < AE; ++i) {
            const int e = tid + i * NT;
            if (e < BM * BK) {
                int mm, kk;
                if (tA) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
                As[(buf * BK + kk) * LDA_S + mm] = ra[i];
            }
        }
    };
    auto storeB = [&](int buf) {
#pragma unroll
        for (int i = 0; i < BE; ++i) {
            const int e = tid + i * NT;
            if (e < BN * BK) {
                int nn, kk;
                if (tB) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
                Bs[(buf * BK + kk) * LDB_S + nn] = rb[i];
            }
        }
    };

    V acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = mk<T>(0, 0);

    const int nk = (Ke + BK - 1) / BK;
    loadA(0);
    loadB(0);
    storeA(0);
    storeB(0);
    __syncthreads();
    for (int t = 0; t < nk; ++t) {
        const int cur = t & 1;
        if (t + 1 < nk) {
            loadA((t + 1) * BK);
            loadB((t + 1) * BK);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            V a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[(cur * BK + kk) * LDA_S + ty + i * TY];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[(cur * BK + kk) * LDB_S + tx + j * TX];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) cfma(acc[i][j], a[i], b[j]);
        }
        if (t + 1 < nk) {
            storeA(cur ^ 1);
            storeB(cur ^ 1);
        }
        __syncthreads();
    }
    const bool use_beta = (beta.x != (T)0) || (beta.y != (T)0);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int gm = m0 + ty + i * TY;
        if (gm >= Me) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int gn = n0 + tx + j * TX;
            if (gn >= Ne) continue;
            V r = cmul(alpha, acc[i][j]);
            if (use_beta) cfma(r, beta, C[(long)gm * ldc + gn]);
            C[(long)gm * ldc + gn] = r;
        }
    }
}

// Products with at most four right-hand columns and A read by rows (op N or
// R): a warp per row of C, the lanes striding the reduction (coalesced rows of
// A), a warp sum per column.  Rows past the run-time count are not written.
constexpr int ROWDOT_NB = 4;
template <typename T>
__global__ void __launch_bounds__(256)
k_rowdot(int M, int N, int K, const int* dM, const int* dN, const int* dK, cplx<T> alpha,
         const cplx<T>* __restrict__ A, long lda, long sA, int conjA, const cplx<T>* __restrict__ B, long ldb,
         long sB, cplx<T>* __restrict__ C, long ldc, long sC, const int* skip) {
    typedef cplx<T> V;
    if (skip && *skip) return;
    int Me = M, Ne = N, Ke = K;
    if (dM) Me = min(Me, *dM);
    if (dN) Ne = min(Ne, *dN);
    if (dK) Ke = min(Ke, *dK);
    const int lane = threadIdx.x & 31, row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= Me) return;
    const long s = blockIdx.y;
    const V* a = A + s * sA + (long)row * lda;
    B += s * sB;
    V acc[ROWDOT_NB];
#pragma unroll
    for (int c = 0; c < ROWDOT_NB; ++c) acc[c] = mk<T>(0, 0);
#pragma unroll 4
    for (int k = lane; k < Ke; k += 32) {
        V x = a[k];
        if (conjA) x.y = -x.y;
#pragma unroll
        for (int c = 0; c < ROWDOT_NB; ++c)
            if (c < Ne) cfma(acc[c], x, B[(long)k * ldb + c]);
    }
#pragma unroll
    for (int c = 0; c < ROWDOT_NB; ++c) {
        acc[c].x = warp_sum(acc[c].x);
        acc[c].y = warp_sum(acc[c].y);
    }
    if (lane == 0)
        for (int c = 0; c < Ne; ++c) C[s * sC + (long)row * ldc + c] = cmul(alpha, acc[c]);
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
static tp_status launch(int batch, int M, int N, int K, const int* dM, const int* dN, const int* dK,
                        cplx<T> alpha, const void* A, long lda, long sA, int opA, const void* B, long ldb,
                        long sB, int opB, cplx<T> beta, void* C, long ldc, long sC, const int* skip,
                        cudaStream_t st) {
    constexpr int NT = (BM / TM) * (BN / TN);
    const size_t smem = (size_t)2 * BK * ((BM + 1) + (BN + 1)) * sizeof(cplx<T>);
    auto kern = k_cgemm<T, BM, BN, BK, TM, TN>;
    if (smem_optin((const void*)kern, smem) != TP_OK) return TP_ERR_CUDA;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
    prof_begin(TP_KC_GEMM, st);
    kern<<<grid, NT, smem, st>>>(M, N, K, dM, dN, dK, alpha, (const cplx<T>*)A, lda, sA, opA,
                                 (const cplx<T>*)B, ldb, sB, opB, beta, (cplx<T>*)C, ldc, sC, skip);
    return launched(TP_KC_GEMM, st);
}

template <typename T>
tp_status cgemm(int batch, int M, int N, int K, const int* dM, const int* dN, const int* dK, double alpha_re,
                double alpha_im, const void* A, long lda, long sA, int opA, const void* B, long ldb, long sB,
                int opB, double beta_re, double beta_im, void* C, long ldc, long sC, const int* skip,
                cudaStream_t st, int* err, int tc_passes) {
    if (batch <= 0 || M <= 0 || N <= 0) return TP_OK;
    if (batch > 65535 || (M + 127) / 128 > 65535) return TP_ERR_ARG;
    if (sizeof(T) == 4 && alpha_re == 1.0 && alpha_im == 0.0 && beta_re == 0.0 && beta_im == 0.0 && opB == OP_N &&
        !dM && !dN && !dK && K > 0) {
        const tp_status e =
            zgemm_tc(batch, M, N, K, A, lda, sA, opA, B, ldb, sB, C, ldc, sC, skip, err, tc_passes, st);
        if (e != TP_ERR_UNSUPPORTED) return e;
    }
    const cplx<T> al = mk<T>((T)alpha_re, (T)alpha_im), be = mk<T>((T)beta_re, (T)beta_im);
    if (N <= ROWDOT_NB && (opA == OP_N || opA == OP_R) && opB == OP_N && beta_re == 0.0 && beta_im == 0.0) {
        dim3 grid((unsigned)((M + 7) / 8), (unsigned)batch);
        prof_begin(TP_KC_GEMM, st);
        k_rowdot<T><<<grid, 256, 0, st>>>(M, N, K, dM, dN, dK, al, (const cplx<T>*)A, lda, sA, opA == OP_R ? 1 : 0,
                                          (const cplx<T>*)B, ldb, sB, (cplx<T>*)C, ldc, sC, skip);
        return launched(TP_KC_GEMM, st);
    }
    if (N <= 16)
        return launch<T, 128, 16, (sizeof(T) == 4 ? 16 : 8), 4, 2>(batch, M, N, K, dM, dN, dK, al, A, lda, sA, opA,
                                                                    B, ldb, sB, opB, be, C, ldc, sC, skip, st);
    return launch<T, 64, 64, (sizeof(T) == 4 ? 16 : 8), 4, 4>(batch, M, N, K, dM, dN, dK, al, A, lda, sA, opA, B,
                                                               ldb, sB, opB, be, C, ldc, sC, skip, st);
}

template tp_status cgemm<float>(int, int, int, int, const int*, const int*, const int*, double, double, const void*,
                                long, long, int, const void*, long, long, int, double, double, void*, long, long,
                                const int*, cudaStream_t, int*, int);
template tp_status cgemm<double>(int, int, int, int, const int*, const int*, const int*, double, double,
                                 const void*, long, long, int, const void*, long, long, int, double, double, void*,
                                 long, long, const int*, cudaStream_t, int*, int);

}  // namespace tp
