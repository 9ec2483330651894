// RT-tSVD (Section 4.2): Algorithm 3 in block form on the half spectrum, the
// full tSVD of Bt by one-sided Jacobi, and truncation by the discrepancy
// principle starting at k_init = r - p (Eq. (kinit)).
//
// Per Fourier slice s (h = n/2+1 of them; slices n-s are conjugates and are
// never formed) the sketch keeps
//   Q   (r x l, vector-major)  orthonormal range basis        (Algorithm 3's Q)
//   QG  (r x m, vector-major)  orthonormal basis of Bt^H = A^H Q
//   R   (r x r)                Bt^H = QG R, built block by block
// so that the SVD of Bt^H = V S U^H comes from the SVD of the small R:
// one-sided Jacobi on R gives R J = U_R S, hence U = J and V = QG U_R.
// Only U^H (Q^H b) is needed, so J itself is never stored: the rotations are
// applied to d = Q^H b as they are made.
#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace tp {

constexpr int JAC_THREADS = 512;
constexpr int MAX_BLOCK = 32;

// ---------------------------------------------------------------------------
// Block orthonormalisation (Algorithm 3, Normalize + reorthogonalisation, in
// block form), one CTA of 1024 threads per Fourier slice:
//   1. Y <- Y - Q (Q^H Y), twice (classical Gram-Schmidt against the basis);
//   2. Y = Q_new R by shifted Cholesky-QR3 (Fukaya et al., 2020): one Cholesky
//      QR of the Gram matrix shifted by 11 (L b + b(b+1)) u ||Y||_F^2, then two
//      plain Cholesky QR passes.  R is upper triangular with a positive real
//      diagonal, so in exact arithmetic Q_new is the Gram-Schmidt basis (the
//      QR factorisation with that normalisation is unique); a zero column
//      (zero pivot) stays zero, as Normalize's breakdown branch gives.
// Y is L x b row-major per slice (b <= BB).  Optional outputs: the basis rows
// r_prev .. r_prev+b-1 (vector-major), the block column of R (coefficients
// against the earlier basis above, the in-block R below, zeros further down to
// row r_rows), and the float64 squared norm of the input block.
// ---------------------------------------------------------------------------
constexpr int ORTH2_GROUPS = 4;  // column groups in the update phase
// threads per CTA: as many as the register footprint of BB accumulators allows
template <typename T, int BB> struct OrthThreads {
    static constexpr int v = (sizeof(T) == 8 && BB == 32) ? 256 : 512;
};

// 1/sqrt(x) for positive normal x: one Newton-Raphson step on the hardware
// approximation (float), y <- y (3 - x y^2) / 2, about one ulp.
template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) {
    const float y = rsqrtf(x);
    return y * fmaf(-0.5f * x * y, y, 1.5f);
}
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }

// Cholesky factor of a 16 x 16 Hermitian Gram matrix (upper triangle of G in
// shared memory) by the first 160 threads (warps 0-4, named barrier 1): thread
// e < 136 holds the upper-triangle entry (i, j), i <= j, in registers.  At step
// k the owner of (k, k) forms the pivot (its reciprocal square root
// Newton-refined), the owners of row k scale it into R[k][.], and every entry
// below row k takes its trailing update from that row.  Each entry sees the
// same operations in the same order as in a column-per-lane Cholesky, with far
// less code per step (the kernel's instruction footprint is what a cold launch
// pays for).  Rows k >= b and zero pivots give zero rows (a zero column stays
// zero).  On the first pass (may_shift) a pivot below 100 u of the largest
// diagonal entry restarts on G + shift I and asks for one more pass (shifted
// CholQR3).  Writes R (row-major, lower part zero) and 1/diag.
__device__ __forceinline__ void bar_chol() { asm volatile("bar.sync 1, 160;" ::: "memory"); }

template <typename T>
__device__ void chol16_par(const cplx<T>* G, cplx<T>* Rk, T* invd, int b, T shift, bool may_shift,
                           int* need_shift, int* passes) {
    typedef cplx<T> V;
    __shared__ T s_id;
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    const bool own = tid < 136;
    int i = 0, j = 0;
    if (own) {
        int rest = tid;
        while (rest >= 16 - i) {
            rest -= 16 - i;
            ++i;
        }
        j = i + rest;
    }
    T dmax = 0;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) dmax = fmax(dmax, G[kk * 16 + kk].x);
#pragma unroll 1
    for (int attempt = 0; attempt < 2; ++attempt) {
        V g = mk<T>(0, 0);
        if (own) {
            g = G[i * 16 + j];
            if (attempt == 1 && i == j) g.x += shift;
            if (i < j) Rk[j * 16 + i] = mk<T>(0, 0);
        }
        if (tid == 0) s_bad = 0;
        bar_chol();
#pragma unroll 1
        for (int k = 0; k < 16; ++k) {
            if (own && i == k && j == k) {
                const T d2 = g.x;
                T d = 0, id = 0;
                if (k < b && d2 < (T)(100.0 * Eps<T>::v) * dmax) s_bad = 1;
                if (k < b && d2 > (T)0) {
                    id = rsqrt_t<T>(d2);
                    d = d2 * id;
                }
                Rk[k * 16 + k] = mk<T>(d, 0);
                invd[k] = id;
                s_id = id;
            }
            bar_chol();
            if (own && i == k && j > k) {
                g = cscale(g, s_id);
                Rk[k * 16 + j] = g;
            }
            bar_chol();
            if (own && i > k) g = csub(g, cmul(cconj(Rk[k * 16 + i]), Rk[k * 16 + j]));
        }
        const bool bad = s_bad != 0;
        if (!may_shift || attempt == 1 || !bad || dmax == (T)0) break;
        bar_chol();
        if (tid == 0) {
            *need_shift = 1;
            *passes += 1;
        }
    }
}


// Row stride (floats) of the partial coefficient tiles of the tensor-core
// products: 32 re/im entries padded to 40, so that the (row g, columns 2t, 2t+1)
// pairs of a half-warp's float2 stores fall on 32 distinct banks.
constexpr int PART_LD = 40;

// ---- float32 Gram matrix on the tensor cores (mma.sync m16n8k8, tf32) -------
// The Gram matrix of a block, C = Y^H Y (a coefficient product with the
// block's own columns as the basis rows), written as a real product with
// interleaved (re, im) reduction indices, each operand split as x = hi + lo in
// tf32 and the products summed as hi*hi + hi*lo + lo*hi (float32-level
// accuracy, as the 3xTF32 products of zgemm_tc; tf32 keeps float32's exponent
// range, so the operands need no scaling).  Within every 8-deep k step lane
// quad member t takes the real indices 2t and 2t+1 (the re and im of one
// complex entry) in the fragment slots t and t+4, the same permutation on both
// operands.
__device__ __forceinline__ uint32_t tf32_bits(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }
__device__ __forceinline__ void split_tf(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_bits(x);
    lo = tf32_bits(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32_16x8x8(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// d += A * [b0; b1] with both split: hi*hi + hi*lo + lo*hi
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], uint32_t b0h,
                                     uint32_t b0l, uint32_t b1h, uint32_t b1l) {
    mma_tf32_16x8x8(d, ah, b0h, b1h);
    mma_tf32_16x8x8(d, ah, b0l, b1l);
    mma_tf32_16x8x8(d, al, b0h, b1h);
}

// Cp (r_prev x 16) = conj(Q) Y for 16 columns of Y (Ys column-major with
// column stride LP, L a multiple of 16); row i of Q starts at Q + i QS, in
// global memory (GQ, read with cache-global loads) or in shared memory.
// Warps take (16-row tile, k range) items; the partial tiles meet in `part`
// (at most 16 x 16 x PART_LD floats) and are summed over the k ranges in a fixed
// order.  Ends with a barrier.
template <bool GQ>
__device__ void orth_coef_mma(const float2* __restrict__ Q, int QS, const float2* Ys, int L, int LP, int r_prev,
                              float2* Cp, float* part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int mt = (r_prev + 15) / 16, nks = L / 4;
    int KC = nw / mt;
    KC = KC < 1 ? 1 : (KC > nks ? nks : KC);
    constexpr uint32_t SGN = 0x80000000u;
    for (int it = warp; it < mt * KC; it += nw) {
        const int mtile = it / KC, kc = it - mtile * KC;
        const int ks0 = kc * nks / KC, ks1 = (kc + 1) * nks / KC;
        const int i0 = mtile * 16 + g, i1 = i0 + 8;
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        for (int ks = ks0; ks < ks1; ++ks) {
            const int e = ks * 4 + t;
            const float2 z = make_float2(0.f, 0.f);
            const float2 q0 = i0 < r_prev ? (GQ ? __ldcg(Q + (long)i0 * QS + e) : Q[(long)i0 * QS + e]) : z;
            const float2 q1 = i1 < r_prev ? (GQ ? __ldcg(Q + (long)i1 * QS + e) : Q[(long)i1 * QS + e]) : z;
            uint32_t ah[4], al[4];
            split_tf(q0.x, ah[0], al[0]);
            split_tf(q1.x, ah[1], al[1]);
            split_tf(q0.y, ah[2], al[2]);
            split_tf(q1.y, ah[3], al[3]);
#pragma unroll
            for (int jh = 0; jh < 2; ++jh) {
                const float2 y = Ys[(jh * 8 + g) * LP + e];
                uint32_t xh, xl, yh, yl;
                split_tf(y.x, xh, xl);
                split_tf(y.y, yh, yl);
                mma3(acc[jh], ah, al, xh, xl, yh, yl);                    // Re: sum Qr Yr + Qi Yi
                mma3(acc[2 + jh], ah, al, yh, yl, xh ^ SGN, xl ^ SGN);    // Im: sum Qr Yi - Qi Yr
            }
        }
        float* P = part + (size_t)kc * mt * 16 * PART_LD;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = mtile * 16 + g + h * 8, col = nt * 8 + 2 * t;
                *(float2*)(P + row * PART_LD + col) = make_float2(acc[nt][2 * h], acc[nt][2 * h + 1]);
            }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < r_prev * 16; idx += blockDim.x) {
        const int i = idx >> 4, j = idx & 15;
        float sr = 0.f, si = 0.f;
        for (int kc = 0; kc < KC; ++kc) {
            const float* P = part + (size_t)kc * mt * 16 * PART_LD + i * PART_LD;
            sr += P[j];
            si += P[16 + j];
        }
        Cp[i * 16 + j] = make_float2(sr, si);
    }
    __syncthreads();
}

// ---- float32 deflation on binary16 tensor cores (mma.sync m16n8k16) -------
// The two products of a classical Gram-Schmidt pass against the basis, with
// every operand split as x = hi + lo in binary16 (11 significant bits each)
// and the products summed as hi*hi + hi*lo + lo*hi in float32: the same
// 22-bit operands as the 3xTF32 split, in half the MMAs (the m16n8k16 form
// takes twice the reduction depth per instruction at the same issue rate).
// binary16 has a narrow exponent range, so both operands are scaled by powers
// of two (exact) before the split and the product scaled back: the basis rows
// are unit vectors (every entry at most 1: x 2^14), the other operand by its
// largest component m, x 2^(13 - floor(log2 m)), which the phase before
// measured.  Components below 2^-17 m keep a subnormal lo part, whose absolute
// error (2^-25 of the scaled unit) is far below the float32 level of the sum.
// Within every 16-deep k step lane quad member t takes the complex entries
// 8s + t (fragment slots 2t, 2t+1: re, im) and 8s + t + 4 (slots 2t+8, 2t+9).
constexpr float H16_QSCALE = 16384.f;  // 2^14

// 2^(13 - floor(log2 m)): m times it lies in [2^13, 2^14); 1 for m = 0 (or NaN)
__device__ __forceinline__ float h16_scale(float m) {
    if (!(m > 0.f)) return 1.f;
    int e = (int)((__float_as_uint(m) >> 23) & 255u) - 127;
    e = e < -100 ? -100 : (e > 113 ? 113 : e);
    return __uint_as_float((unsigned)(127 + 13 - e) << 23);
}
// (a, b) -> binary16 pairs hi = rn(a, b), lo = rn(a - hi_a, b - hi_b); a in the low half
__device__ __forceinline__ void split_h2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 f = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - f.x, b - f.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}
__device__ __forceinline__ void mma_f16_16x8x16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// d += A * [b0; b1] with both split: hi*hi + hi*lo + lo*hi
__device__ __forceinline__ void mmah3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], uint32_t b0h,
                                      uint32_t b0l, uint32_t b1h, uint32_t b1l) {
    mma_f16_16x8x16(d, ah, b0h, b1h);
    mma_f16_16x8x16(d, ah, b0l, b1l);
    mma_f16_16x8x16(d, al, b0h, b1h);
}
// the packed pair (lo16, hi16) -> (hi16, lo16) with the sign of the given half flipped
__device__ __forceinline__ uint32_t swap_neg(uint32_t x, uint32_t sign) { return __byte_perm(x, 0, 0x1032) ^ sign; }
// largest value of v over the warp, written to wmax[warp] by lane 0
__device__ __forceinline__ void warp_max_to(float v, float* wmax) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
}
__device__ __forceinline__ float max_of(const float* wmax, int n) {
    float m = 0.f;
    for (int w = 0; w < n; ++w) m = fmaxf(m, wmax[w]);
    return m;
}

// Cp (r_prev x 16) = conj(Q) Y for the 16 columns of Y (Ys column-major with
// column stride LP, L a multiple of 16); row i of Q (a unit vector) starts at
// Q + i L in global memory (cache-global loads).  ymax: the largest component
// of Y.  Warps take (16-row tile, k range) items; the partial tiles, scaled
// back, meet in `part` and are summed over the k ranges in a fixed order.
// The largest component of Cp goes to cmax_w (one entry per warp).  Ends with
// a barrier.
__device__ void orth_coef_h16(const float2* __restrict__ Q, const float2* Ys, int L, int LP, int r_prev, float ymax,
                              float2* Cp, float* part, float* cmax_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int mt = (r_prev + 15) / 16, nks = L / 8;
    int KC = nw / mt;
    KC = KC < 1 ? 1 : (KC > nks ? nks : KC);
    const float sy = h16_scale(ymax), back = 1.f / (H16_QSCALE * sy);
    constexpr uint32_t HI = 0x80000000u;
    for (int it = warp; it < mt * KC; it += nw) {
        const int mtile = it / KC, kc = it - mtile * KC;
        const int ks0 = kc * nks / KC, ks1 = (kc + 1) * nks / KC;
        const int i0 = mtile * 16 + g, i1 = i0 + 8;
        const bool ok0 = i0 < r_prev, ok1 = i1 < r_prev;
        const float2* q0 = Q + (long)i0 * L;
        const float2* q1 = Q + (long)i1 * L;
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
        for (int ks = ks0; ks < ks1; ++ks) {
            const int e0 = ks * 8 + t, e1 = e0 + 4;
            const float2 z = make_float2(0.f, 0.f);
            const float2 a0 = ok0 ? __ldcg(q0 + e0) : z, a1 = ok1 ? __ldcg(q1 + e0) : z;
            const float2 a2 = ok0 ? __ldcg(q0 + e1) : z, a3 = ok1 ? __ldcg(q1 + e1) : z;
            uint32_t ah[4], al[4];
            split_h2(a0.x * H16_QSCALE, a0.y * H16_QSCALE, ah[0], al[0]);
            split_h2(a1.x * H16_QSCALE, a1.y * H16_QSCALE, ah[1], al[1]);
            split_h2(a2.x * H16_QSCALE, a2.y * H16_QSCALE, ah[2], al[2]);
            split_h2(a3.x * H16_QSCALE, a3.y * H16_QSCALE, ah[3], al[3]);
#pragma unroll
            for (int jh = 0; jh < 2; ++jh) {
                const float2 y0 = Ys[(jh * 8 + g) * LP + e0], y1 = Ys[(jh * 8 + g) * LP + e1];
                uint32_t r0h, r0l, r1h, r1l;
                split_h2(y0.x * sy, y0.y * sy, r0h, r0l);
                split_h2(y1.x * sy, y1.y * sy, r1h, r1l);
                // Re: sum qr yr + qi yi with (yr, yi); Im: sum qr yi - qi yr with (yi, -yr)
                mmah3(acc[jh], ah, al, r0h, r0l, r1h, r1l);
                mmah3(acc[2 + jh], ah, al, swap_neg(r0h, HI), swap_neg(r0l, HI), swap_neg(r1h, HI),
                      swap_neg(r1l, HI));
            }
        }
        float* P = part + (size_t)kc * mt * 16 * PART_LD;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = mtile * 16 + g + h * 8, col = nt * 8 + 2 * t;
                *(float2*)(P + row * PART_LD + col) = make_float2(acc[nt][2 * h] * back, acc[nt][2 * h + 1] * back);
            }
    }
    __syncthreads();
    float cm = 0.f;
    for (int idx = threadIdx.x; idx < r_prev * 16; idx += blockDim.x) {
        const int i = idx >> 4, j = idx & 15;
        float sr = 0.f, si = 0.f;
        for (int kc = 0; kc < KC; ++kc) {
            const float* P = part + (size_t)kc * mt * 16 * PART_LD + i * PART_LD;
            sr += P[j];
            si += P[16 + j];
        }
        Cp[i * 16 + j] = make_float2(sr, si);
        cm = fmaxf(cm, fmaxf(fabsf(sr), fabsf(si)));
    }
    warp_max_to(cm, cmax_w);
    __syncthreads();
}

// Ys (L x 16, column-major, column stride LP) -= Q^T Cp (Q's rows are the
// basis vectors; no conjugation): a warp per 16-row tile of Y.  L a multiple
// of 16; cmax: the largest component of Cp.  The largest component of the
// updated Y goes to ymax_w (one entry per warp).
__device__ void orth_update_h16(const float2* __restrict__ Q, float2* Ys, int L, int LP, int r_prev,
                                const float2* Cp, float cmax, float* ymax_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int mt = L / 16, nks = (r_prev + 7) / 8;
    const float sc = h16_scale(cmax), back = 1.f / (H16_QSCALE * sc);
    constexpr uint32_t LO = 0x00008000u;
    float ym = 0.f;
    for (int mtile = warp; mtile < mt; mtile += nw) {
        const int e0 = mtile * 16 + g, e1 = e0 + 8;
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
        for (int ks = 0; ks < nks; ++ks) {
            const int i0 = ks * 8 + t, i1 = i0 + 4;
            const bool ok0 = i0 < r_prev, ok1 = i1 < r_prev;
            const float2 z = make_float2(0.f, 0.f);
            const float2 a0 = ok0 ? __ldcg(Q + (long)i0 * L + e0) : z, a1 = ok0 ? __ldcg(Q + (long)i0 * L + e1) : z;
            const float2 a2 = ok1 ? __ldcg(Q + (long)i1 * L + e0) : z, a3 = ok1 ? __ldcg(Q + (long)i1 * L + e1) : z;
            uint32_t ah[4], al[4];
            split_h2(a0.x * H16_QSCALE, a0.y * H16_QSCALE, ah[0], al[0]);
            split_h2(a1.x * H16_QSCALE, a1.y * H16_QSCALE, ah[1], al[1]);
            split_h2(a2.x * H16_QSCALE, a2.y * H16_QSCALE, ah[2], al[2]);
            split_h2(a3.x * H16_QSCALE, a3.y * H16_QSCALE, ah[3], al[3]);
#pragma unroll
            for (int jh = 0; jh < 2; ++jh) {
                const float2 c0 = ok0 ? Cp[i0 * 16 + jh * 8 + g] : z, c1 = ok1 ? Cp[i1 * 16 + jh * 8 + g] : z;
                uint32_t r0h, r0l, r1h, r1l;
                split_h2(c0.x * sc, -c0.y * sc, r0h, r0l);
                split_h2(c1.x * sc, -c1.y * sc, r1h, r1l);
                // Re: sum qr cr - qi ci with (cr, -ci); Im: sum qr ci + qi cr with (ci, cr)
                mmah3(acc[jh], ah, al, r0h, r0l, r1h, r1l);
                mmah3(acc[2 + jh], ah, al, swap_neg(r0h, LO), swap_neg(r0l, LO), swap_neg(r1h, LO),
                      swap_neg(r1l, LO));
            }
        }
#pragma unroll
        for (int jh = 0; jh < 2; ++jh)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int row = (c >> 1) ? e1 : e0, j = jh * 8 + 2 * t + (c & 1);
                float2* y = Ys + j * LP + row;
                const float2 v = make_float2(y->x - acc[jh][c] * back, y->y - acc[2 + jh][c] * back);
                *y = v;
                ym = fmaxf(ym, fmaxf(fabsf(v.x), fabsf(v.y)));
            }
    }
    warp_max_to(ym, ymax_w);
}

// Shared-memory extents of k_orth beyond its matrices: the partial tiles of
// the tensor-core deflation (float32, 16 columns) and the Gram partials (one
// per thread, at least one per upper-triangle entry).
template <typename T, int BB> constexpr size_t orth_part_bytes() {
    return (sizeof(T) == 4 && BB == 16) ? (size_t)16 * 16 * PART_LD * sizeof(float) : 0;
}
template <typename T, int BB> constexpr size_t orth_gram_elems() {
    return (size_t)(BB * (BB + 1) / 2 > OrthThreads<T, BB>::v ? BB * (BB + 1) / 2 : OrthThreads<T, BB>::v);
}

template <typename T, int BB>
__global__ void __launch_bounds__(OrthThreads<T, BB>::v)
k_orth(cplx<T>* Y, long sY, int L, int b, const cplx<T>* Qb, long sQ, int r_prev, cplx<T>* Qout,
       cplx<T>* R, long ldr, long sR, int r_rows, double* normsq, const int* skip, int final_pass, State* eta,
       int n_dft, int r_new) {
    typedef cplx<T> V;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    // Ys[j*LP + row], BB columns (unused ones zero); the odd column stride LP = L + 1
    // keeps the column-parallel accesses (load, write-back, tensor-core operand
    // reads) free of shared-memory bank conflicts
    const int LP = L + 1;
    V* Ys = (V*)smraw;
    V* Cs = Ys + (size_t)BB * LP;           // r_prev x BB, summed over both passes
    V* Cp = Cs + (size_t)r_prev * BB;       // r_prev x BB, this pass
    V* G = Cp + (size_t)r_prev * BB;        // BB x BB Gram / Cholesky work
    V* Rk = G + BB * BB;                    // this pass's R
    V* Ra = Rk + BB * BB;                   // accumulated in-block R
    V* Rt = Ra + BB * BB;                   // scratch for the product
    float* part = (float*)(Rt + BB * BB);   // tensor-core deflation: partial coefficient tiles
    V* gpart = (V*)((unsigned char*)part + orth_part_bytes<T, BB>());  // Gram partials
    __shared__ double red[33];
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = OrthThreads<T, BB>::v / 32;
    Y += (long)s * sY;

    __shared__ int passes, need_shift;
    if (tid == 0) {  // published by the barriers of the norm below
        passes = final_pass ? 2 : 1;
        need_shift = 0;
    }
    T nn = 0;
    float ymax = 0.f;  // largest component of the block (binary16 deflation scale)
    {
        // Y row-major L x b: coalesced reads, eight per thread in flight
        constexpr int U = 8;
        const int tot = L * b, nt = blockDim.x;
        for (int e0 = tid; e0 < tot; e0 += U * nt) {
            V v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * nt;
                v[u] = e < tot ? Y[e] : mk<T>(0, 0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * nt;
                if (e < tot) {
                    const int row = e / b, j = e - row * b;
                    Ys[j * LP + row] = v[u];
                    nn += cabs2(v[u]);
                    ymax = fmaxf(ymax, fmaxf(fabsf((float)v[u].x), fabsf((float)v[u].y)));
                }
            }
        }
    }
    for (int e = tid; e < L * (BB - b); e += blockDim.x) {
        const int j = b + e / L, row = e - (j - b) * L;
        Ys[j * LP + row] = mk<T>(0, 0);
    }
    for (int e = tid; e < BB * BB; e += blockDim.x) Ra[e] = mk<T>((e / BB) == (e % BB) ? (T)1 : (T)0, 0);
    __shared__ float wmax_y[32], wmax_c[32];  // per-warp maxima of |Y| and |Cp| components
    warp_max_to(ymax, wmax_y);                 // published by the barriers of the norm
    const double nnd = block_sum_t(nn, red);
    if (normsq && tid == 0) normsq[s] = nnd;

    // 1. two CGS passes against the basis (one for intermediate blocks of the
    //    power iteration: the kept block after them gets two)
    if (r_prev > 0) {
        const V* Q = Qb + (long)s * sQ;
        const int dpasses = final_pass ? 2 : 1;
        const bool tc = sizeof(T) == 4 && BB == 16 && (L & 15) == 0 && r_prev <= 256;  // part: 16 row tiles
        for (int pass = 0; pass < dpasses; ++pass) {
          if (tc) {
            orth_coef_h16((const float2*)Q, (const float2*)Ys, L, LP, r_prev, max_of(wmax_y, NW), (float2*)Cp,
                          part, wmax_c);
            orth_update_h16((const float2*)Q, (float2*)Ys, L, LP, r_prev, (const float2*)Cp, max_of(wmax_c, NW),
                            wmax_y);
          } else {
            // two basis vectors per warp share every shared-memory read of Y
            for (int i0 = 2 * warp; i0 < r_prev; i0 += 2 * NW) {
                const bool two = i0 + 1 < r_prev;
                V acc0[BB], acc1[BB];
#pragma unroll
                for (int j = 0; j < BB; ++j) acc0[j] = acc1[j] = mk<T>(0, 0);
                const V* qa = Q + (long)i0 * L;
                const V* qb = two ? qa + L : qa;
                int row = lane;
                for (; row + 32 < L; row += 64) {
                    const V a0 = qa[row], a1 = qa[row + 32];
                    V b0 = qb[row], b1 = qb[row + 32];
                    if (!two) b0 = b1 = mk<T>(0, 0);
#pragma unroll
                    for (int j = 0; j < BB; ++j) {
                        const V y0 = Ys[j * LP + row], y1 = Ys[j * LP + row + 32];
                        cfmac(acc0[j], a0, y0);
                        cfmac(acc1[j], b0, y0);
                        cfmac(acc0[j], a1, y1);
                        cfmac(acc1[j], b1, y1);
                    }
                }
                for (; row < L; row += 32) {
                    const V a0 = qa[row];
                    const V b0 = two ? qb[row] : mk<T>(0, 0);
#pragma unroll
                    for (int j = 0; j < BB; ++j) {
                        const V y0 = Ys[j * LP + row];
                        cfmac(acc0[j], a0, y0);
                        cfmac(acc1[j], b0, y0);
                    }
                }
                const int col = (BB == 32) ? lane : (lane >> 1);
                const V t0 = warp_reduce_scatter<V, BB>(acc0);
                if ((BB == 32 || (lane & 1) == 0)) Cp[(size_t)i0 * BB + col] = t0;
                const V t1 = warp_reduce_scatter<V, BB>(acc1);
                if (two && (BB == 32 || (lane & 1) == 0)) Cp[(size_t)(i0 + 1) * BB + col] = t1;
            }
            __syncthreads();
            constexpr int CPG = BB / ORTH2_GROUPS;
            for (int e = tid; e < L * ORTH2_GROUPS; e += blockDim.x) {
                const int g = e / L, row = e - g * L;
                V acc[CPG];
#pragma unroll
                for (int c = 0; c < CPG; ++c) acc[c] = mk<T>(0, 0);
                int i = 0;
                for (; i + 3 < r_prev; i += 4) {  // four loads in flight per thread
                    const V q0 = Q[(long)i * L + row], q1 = Q[(long)(i + 1) * L + row];
                    const V q2 = Q[(long)(i + 2) * L + row], q3 = Q[(long)(i + 3) * L + row];
#pragma unroll
                    for (int c = 0; c < CPG; ++c) {
                        const V* cp = Cp + (size_t)i * BB + g * CPG + c;
                        cfma(acc[c], q0, cp[0]);
                        cfma(acc[c], q1, cp[BB]);
                        cfma(acc[c], q2, cp[2 * BB]);
                        cfma(acc[c], q3, cp[3 * BB]);
                    }
                }
                for (; i < r_prev; ++i) {
                    const V q = Q[(long)i * L + row];
#pragma unroll
                    for (int c = 0; c < CPG; ++c) cfma(acc[c], q, Cp[(size_t)i * BB + g * CPG + c]);
                }
#pragma unroll
                for (int c = 0; c < CPG; ++c) {
                    V* y = Ys + (g * CPG + c) * LP + row;
                    *y = csub(*y, acc[c]);
                }
            }
          }
            for (int e = tid; e < r_prev * BB; e += blockDim.x) Cs[e] = pass ? cadd(Cs[e], Cp[e]) : Cp[e];
            __syncthreads();
        }
    }

    // 2. Cholesky QR of the block: CholQR2 when the first Gram matrix is well
    //    conditioned, otherwise shifted CholQR3 (a shifted first pass, then two
    //    plain passes).  G holds the Gram matrix, Rk this pass's R, Rt = Rk^-1,
    //    Ra the accumulated in-block R (only when R is an output).
    __shared__ T invd[BB];
    // Intermediate blocks (inside the power iteration) only need a
    // well-conditioned basis of the right subspace: one Cholesky QR pass
    // (`passes` set at the start).  Blocks that are kept (Q, QG, R) get two.
    T shift = 0;  // the shifted first pass's shift (Cholesky warp only)
    for (int pass = 0; pass < passes; ++pass) {
        // Gram matrix: float32 with 16 columns on the tensor cores (the
        // coefficient product with the block's own columns as the basis, the
        // full 16 x 16, 3xTF32); otherwise the upper triangle incl. diagonal by
        // a thread per (entry, chunk of rows), the chunk sums meeting in gpart
        if (sizeof(T) == 4 && BB == 16 && (L & 15) == 0) {
            orth_coef_mma<false>((const float2*)Ys, LP, (const float2*)Ys, L, LP, 16, (float2*)G, part);
        } else {
            constexpr int NE = BB * (BB + 1) / 2;
            const int nch = (int)blockDim.x / NE > 1 ? (int)blockDim.x / NE : 1;
            const int rpc = (L + nch - 1) / nch;
            for (int it = tid; it < NE * nch; it += blockDim.x) {
                const int c = it / NE, e = it - c * NE;
                int i = 0, rest = e;
                while (rest >= BB - i) {
                    rest -= BB - i;
                    ++i;
                }
                const V* yi = Ys + i * LP;
                const V* yj = Ys + (i + rest) * LP;
                const int r0 = c * rpc, r1 = min(L, r0 + rpc);
                V acc = mk<T>(0, 0);
#pragma unroll 4
                for (int row = r0; row < r1; ++row) cfmac(acc, yi[row], yj[row]);
                gpart[it] = acc;
            }
            __syncthreads();
            for (int e = tid; e < NE; e += blockDim.x) {
                int i = 0, rest = e;
                while (rest >= BB - i) {
                    rest -= BB - i;
                    ++i;
                }
                V acc = gpart[e];
                for (int c = 1; c < nch; ++c) acc = cadd(acc, gpart[c * NE + e]);
                G[i * BB + i + rest] = acc;
            }
        }
        __syncthreads();
        __shared__ T s_shift;
        if (pass == 0 && warp == 0) {
            // 11 (L b + b(b+1)) u ||Y||_F^2, ||Y||_F^2 the trace of the Gram matrix
            T y2 = lane < BB ? G[lane * BB + lane].x : (T)0;
            y2 = warp_sum(y2);
            shift = (T)(11.0 * ((double)L * b + (double)b * (b + 1)) * Eps<T>::v) * y2;
            if (lane == 0) s_shift = shift;
        }
        if (BB == 16 && sizeof(T) == 4) {
            if (tid < 160) {
                bar_chol();  // s_shift
                chol16_par<T>(G, Rk, invd, b, s_shift, pass == 0, &need_shift, &passes);
            }
        } else if (warp == 0) {
            // Cholesky G (+ shift) = R^H R by the first warp: at step k the
            // lanes form row k of R, then update the trailing Gram entries as
            // independent (i, j) pairs.  A zero pivot gives a zero row (a zero
            // column stays zero).  The first pass retries with the shift when a
            // pivot falls below 100 u of the largest diagonal entry.
            T dmax = 0;
            for (int k = 0; k < BB; ++k) dmax = fmax(dmax, G[k * BB + k].x);
            for (int attempt = 0; attempt < 2; ++attempt) {
                const bool shifted = attempt == 1;
                if (shifted) {
                    // restore the Gram matrix from its untouched copy in Rt, add the shift
                    for (int e = lane; e < BB * BB; e += 32) G[e] = Rt[e];
                    __syncwarp();
                    if (lane < BB) G[lane * BB + lane].x += (T)shift;
                } else {
                    for (int e = lane; e < BB * BB; e += 32) Rt[e] = G[e];
                }
                __syncwarp();
                bool bad = false;
                for (int k = 0; k < BB; ++k) {
                    const T d2 = G[k * BB + k].x;
                    if (k < b && d2 < (T)(100.0 * Eps<T>::v) * dmax) bad = true;
                    const T d = (k < b && d2 > (T)0) ? sqrt(d2) : (T)0;
                    const T id = d > (T)0 ? (T)1 / d : (T)0;
                    const int j = lane;
                    if (j < BB) {
                        V v = mk<T>(0, 0);
                        if (j > k) v = cscale(G[k * BB + j], id);
                        else if (j == k) v = mk<T>(d, 0);
                        Rk[k * BB + j] = v;
                    }
                    if (lane == 0) invd[k] = id;
                    __syncwarp();
                    // trailing update G[i][jj] -= conj(R[k][i]) R[k][jj], k < i <= jj:
                    // a half-warp (BB = 16) or a warp (BB = 32) per row i, lane
                    // offset jj - i (no integer division)
                    constexpr int RW = BB == 16 ? 16 : 32;
                    const int rsub = lane / RW, jo = lane % RW;
                    for (int i = k + 1 + rsub; i < BB; i += 32 / RW) {
                        const int jj = i + jo;
                        if (jj < BB)
                            G[i * BB + jj] = csub(G[i * BB + jj], cmul(cconj(Rk[k * BB + i]), Rk[k * BB + jj]));
                    }
                    __syncwarp();
                }
                if (pass > 0 || shifted || !bad || dmax == (T)0) break;
                if (lane == 0) {
                    need_shift = 1;
                    passes += 1;
                }
            }
        }
        __syncthreads();
        // Y <- Y R^{-1}: per row, forward substitution (diagonal reciprocals
        // precomputed); the threads beyond the rows meanwhile form the
        // accumulated in-block R' = Rk Ra when R is an output
        for (int row = tid; row < L; row += blockDim.x) {
            V x[BB];
#pragma unroll
            for (int jj = 0; jj < BB; ++jj) {
                V y = Ys[jj * LP + row];
#pragma unroll
                for (int i = 0; i < jj; ++i) y = csub(y, cmul(x[i], Rk[i * BB + jj]));
                x[jj] = cscale(y, invd[jj]);
            }
#pragma unroll
            for (int jj = 0; jj < BB; ++jj) Ys[jj * LP + row] = x[jj];
        }
        if (R) {
            const int nthr = (int)blockDim.x, t0 = L < nthr ? L : 0;  // threads idle in the solve when L < blockDim
            for (int e = tid - t0; e >= 0 && e < BB * BB; e += nthr - t0) {
                const int i = e / BB, jj = e - i * BB;
                V acc = mk<T>(0, 0);
                for (int t = i; t <= jj; ++t) cfma(acc, Rk[i * BB + t], Ra[t * BB + jj]);
                Rt[e] = (i <= jj) ? acc : mk<T>(0, 0);
            }
        }
        __syncthreads();
        if (R) {  // the product becomes the accumulated R (swap the two buffers)
            V* tmp = Ra;
            Ra = Rt;
            Rt = tmp;
        }
    }

    for (int e = tid; e < L * b; e += blockDim.x) {
        const int row = e / b, j = e - row * b;
        Y[e] = Ys[j * LP + row];
    }
    if (Qout) {
        V* Qo = Qout + (long)s * sQ + (long)r_prev * L;
        for (int e = tid; e < L * b; e += blockDim.x) {
            const int j = e / L, row = e - j * L;
            Qo[e] = Ys[j * LP + row];
        }
    }
    if (R) {
        V* Rs = R + (long)s * sR;
        for (int e = tid; e < r_rows * b; e += blockDim.x) {
            const int i = e / b, j = e - i * b;
            V v = mk<T>(0, 0);  // rows below this block stay zero: R is block upper triangular
            if (i < r_prev) v = Cs[(size_t)i * BB + j];
            else if (i < r_prev + b) v = Ra[(i - r_prev) * BB + j];
            Rs[(long)i * ldr + r_prev + j] = v;
        }
    }
    if (eta) {
        // the last CTA to finish takes the eta update of Algorithm 3 for the
        // block (eta <- eta - ||Bt(block)||_F^2, Parseval-weighted over the
        // slices, in the fixed order of 256 partial sums), sets r and the stop
        // flag, and resets the arrival count for the next block
        __shared__ int last;
        __threadfence();
        __syncthreads();
        if (tid == 0) last = atomicAdd(&eta->arrived, 1u) == gridDim.x - 1;
        __syncthreads();
        if (last) {
            __threadfence();
            double a = 0.0;
            if (tid < 256)
                for (int s2 = tid; s2 < (int)gridDim.x; s2 += 256) a += parseval_w(s2, n_dft) * __ldcg(&normsq[s2]);
            a = block_sum(a, red);
            if (tid == 0) {
                eta->eta -= a / (double)n_dft;
                eta->r = r_new;
                if (eta->eta < eta->eps2) eta->done = 1;
                eta->arrived = 0;
            }
        }
    }
}

static size_t orth_smem(int L, int b, int r_prev, size_t c) {
    const size_t BB = b <= 16 ? 16 : 32;
    const size_t part = c == 8 ? (BB == 16 ? orth_part_bytes<float, 16>() : orth_part_bytes<float, 32>())
                               : (BB == 16 ? orth_part_bytes<double, 16>() : orth_part_bytes<double, 32>());
    const size_t gram = c == 8 ? (BB == 16 ? orth_gram_elems<float, 16>() : orth_gram_elems<float, 32>())
                               : (BB == 16 ? orth_gram_elems<double, 16>() : orth_gram_elems<double, 32>());
    return ((size_t)BB * (L + 1) + 2 * (size_t)r_prev * BB + 4 * BB * BB + gram) * c + part;
}

template <typename T>
static tp_status orth(int h, cplx<T>* Y, long sY, int L, int b, const cplx<T>* Qb, long sQ, int r_prev,
                      cplx<T>* Qout, cplx<T>* R, long ldr, long sR, int r_rows, double* normsq, const int* skip,
                      cudaStream_t st, State* eta = nullptr, int n_dft = 0, int r_new = 0) {
    const int final_pass = (Qout != nullptr || R != nullptr) ? 1 : 0;
    const size_t smem = orth_smem(L, b, r_prev, sizeof(cplx<T>));
    auto kern = b <= 16 ? k_orth<T, 16> : k_orth<T, 32>;
    const int nt = b <= 16 ? OrthThreads<T, 16>::v : OrthThreads<T, 32>::v;
    if (smem_optin((const void*)kern, smem) != TP_OK) return TP_ERR_CUDA;
    prof_begin(TP_KC_ORTH, st);
    kern<<<h, nt, smem, st>>>(Y, sY, L, b, Qb, sQ, r_prev, Qout, R, ldr, sR, r_rows, normsq, skip, final_pass, eta,
                              n_dft, r_new);
    return launched(TP_KC_ORTH, st);
}

// ---------------------------------------------------------------------------
// Scalars: ||A||^2 from the DFT partials and eps^2 (the eta update of
// Algorithm 3 is taken by the last CTA of each block's k_orth launch).
// ---------------------------------------------------------------------------
__device__ double fixed_order_sum(const double* v, int count, double* red) {
    double a = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) a += v[i];
    return block_sum(a, red);
}

__global__ void k_rt_init(State* st, const double* partsA, int nA, const double* partsB, int nB, double eps,
                          double eps_rel, int n) {
    __shared__ double red[32];
    const double a2 = fixed_order_sum(partsA, nA, red);
    const double b2 = fixed_order_sum(partsB, nB, red);
    if (threadIdx.x == 0) {
        st->norm_a2 = a2;
        st->norm_b2 = b2;
        st->eta = a2;
        // eps < 0: sketch to r_max whatever eta (the T-tSVD form); eps2 = -1 never stops it
        st->eps2 = eps > 0.0 ? eps * eps : (eps < 0.0 ? -1.0 : eps_rel * eps_rel * a2);
        st->done = (st->eta < st->eps2) ? 1 : 0;
        st->r = 0;
        st->k = 0;
        st->status = TP_OK;
        st->sweeps = 0;
        st->sigma_max = 0.0;
        st->arrived = 0;
        st->nonfinite = (isfinite(a2) && isfinite(b2)) ? 0 : 1;
    }
}

// ---------------------------------------------------------------------------
// One-sided Jacobi SVD of R (r x r) per slice, rotations from the right
// (cyclic round-robin ordering, r/2 disjoint pairs per round, a group of
// lanes per pair: 8 in the float32 register form, 16 in the shared-memory
// form).  Tracks d' = J^H d.  Outputs, sorted by decreasing sigma:
// sigma (r), U_R (r x r row-major, columns normalised), d'.
//
// A pair (p, q) with Gram entries a = |x|^2, b = |y|^2, g = x^H y is rotated
// when |g| > tol sqrt(a b) (tol = 4 sqrt(r) u): with e = g/|g|,
// zeta = (b - a) / (2|g|), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1/sqrt(1 + t^2), s = c t, the columns become x' = c x - s conj(e) y and
// y' = s x + c conj(e) y, which makes them orthogonal.
// Convergence is quadratic once the columns are nearly orthogonal: a sweep
// whose largest relative off-diagonal |g|/sqrt(a b) is below sqrt(tol) leaves
// residues below tol, so the sweep after it (which would only confirm) is
// skipped.
// ---------------------------------------------------------------------------

// Pair (p, q) of slot kp in round t of the round-robin ordering of rr (even)
// columns; valid only when q < r.
__device__ __forceinline__ bool rr_pair(int t, int kp, int rr, int r, int& p, int& q) {
    p = 0;
    q = 0;
    if (kp == 0) {
        q = 1 + t;
    } else if (kp < rr / 2) {
        p = 1 + (t + kp) % (rr - 1);
        q = 1 + (t - kp + (rr - 1)) % (rr - 1);
    }
    if (p > q) {
        const int x = p;
        p = q;
        q = x;
    }
    return kp < rr / 2 && q < r && p != q;
}

// Sweeps in shared memory with IEEE arithmetic (any precision).
template <typename T>
__device__ int jacobi_sweeps_smem(cplx<T>* Rs, cplx<T>* dp, int np, int r, int max_sweeps, T tol) {
    typedef cplx<T> V;
    __shared__ int rot_count;
    __shared__ int max_off;  // bit pattern of the largest |g| / sqrt(a b) of a sweep (non-negative float)
    const int tid = threadIdx.x, hl = tid & 15, slot = tid >> 4, nslots = blockDim.x >> 4;
    const int rr = r + (r & 1);
    const float stop_off = (float)sqrt((double)tol);
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (tid == 0) {
            rot_count = 0;
            max_off = 0;
        }
        __syncthreads();
        for (int t = 0; t < rr - 1; ++t) {
            for (int base = 0; base < rr / 2; base += nslots) {
                int p, q;
                const bool valid = rr_pair(t, base + slot, rr, r, p, q);
                V* cp = Rs + (size_t)p * r;
                V* cq = Rs + (size_t)q * r;
                T a = 0, bq = 0;
                V g = mk<T>(0, 0);
                if (valid)
                    for (int i = hl; i < r; i += 16) {
                        const V x = cp[i], y = cq[i];
                        a += x.x * x.x + x.y * x.y;
                        bq += y.x * y.x + y.y * y.y;
                        cfmac(g, x, y);
                    }
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    bq += __shfl_xor_sync(0xffffffffu, bq, o);
                    g.x += __shfl_xor_sync(0xffffffffu, g.x, o);
                    g.y += __shfl_xor_sync(0xffffffffu, g.y, o);
                }
                const T ag = sqrt(g.x * g.x + g.y * g.y);
                if (valid && hl == 0 && a > (T)0 && bq > (T)0) {
                    const float rel = (float)(ag / (sqrt(a) * sqrt(bq)));
                    atomicMax(&max_off, __float_as_int(rel));
                }
                if (valid && ag > (T)0 && ag > tol * sqrt(a) * sqrt(bq)) {
                    const T zeta = (bq - a) / ((T)2 * ag);
                    const T tt = (zeta >= (T)0 ? (T)1 : (T)-1) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
                    const T c = (T)1 / sqrt((T)1 + tt * tt), sn = c * tt;
                    const V e = mk<T>(g.x / ag, g.y / ag);
                    const V ec = cconj(e);
                    for (int i = hl; i < r; i += 16) {
                        const V x = cp[i];
                        const V ey = cmul(ec, cq[i]);
                        cp[i] = mk<T>(c * x.x - sn * ey.x, c * x.y - sn * ey.y);
                        cq[i] = mk<T>(sn * x.x + c * ey.x, sn * x.y + c * ey.y);
                    }
                    for (int cc = hl; cc < np; cc += 16) {  // the rows p, q of d' (np right-hand sides)
                        const V x = dp[p * np + cc];
                        const V ey = cmul(e, dp[q * np + cc]);
                        dp[p * np + cc] = mk<T>(c * x.x - sn * ey.x, c * x.y - sn * ey.y);
                        dp[q * np + cc] = mk<T>(sn * x.x + c * ey.x, sn * x.y + c * ey.y);
                    }
                    if (hl == 0) atomicAdd(&rot_count, 1);
                }
            }
            __syncthreads();
        }
        const int rc = rot_count;
        const float mo = __int_as_float(max_off);
        __syncthreads();
        if (rc == 0 || mo < stop_off) return sweep + 1;
    }
    return sweep;  // sweeps executed
}

// 1/sqrt(x) for normal positive x: one Newton-Raphson step on the hardware
// approximation, y <- y (3 - x y^2) / 2, which brings it to about one ulp.
__device__ __forceinline__ float rsqrt_nr(float x) {
    const float y = rsqrtf(x);
    return y * fmaf(-0.5f * x * y, y, 1.5f);
}

// Float32 sweeps with the two columns of a pair held in registers by GL = 8
// lanes (r <= GL EPL; fewer lanes per pair than a half-warp amortise the
// rotation's scalar work and shuffles over more entries per lane, and the
// CTA needs only 512 threads): the Gram entries and the rotation read and
// write shared memory once per element (as 16-byte pairs of entries when r
// is even), the rotation parameters come from Newton-refined reciprocal
// square roots (c^2 + s^2 = 1 to about an ulp), the pair indices of the round-robin ordering advance by
// one per round (no integer division), and the per-round "any rotation" flag
// rides on the round's barrier.
template <int EPL, bool V2, int GL = 8>
__device__ int jacobi_sweeps_reg(float2* Rs, float2* dp, int np, int r, int max_sweeps, float tol, float* cn) {
    __shared__ int max_off2;  // bit pattern of the largest (|g|^2 / (a b)) of a sweep
    const int tid = threadIdx.x, lane = tid & 31, hl = tid & (GL - 1), slot = tid / GL, nslots = blockDim.x / GL;
    const int rr = r + (r & 1), npair = rr / 2;
    const float tol2 = tol * tol;
    // element e of this lane: index hl + GL e, or with pairs (V2) 2 (hl + GL (e / 2)) + e % 2
    auto idx = [&](int e) { return V2 ? 2 * (hl + GL * (e >> 1)) + (e & 1) : hl + GL * e; };
    // squared column norms: recomputed from the columns at the start of every
    // sweep and carried through its rotations (a rotation by t = tan(theta)
    // with |g| the off-diagonal entry leaves |x|^2 - t |g| and |y|^2 + t |g|),
    // so a round forms only g = x^H y (cn: r floats of shared memory)
    const int warp = tid >> 5, nw = blockDim.x >> 5;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (tid == 0) max_off2 = 0;
        for (int j = warp; j < r; j += nw) {
            float sq = 0.f;
            for (int i = lane; i < r; i += 32) {
                const float2 v = Rs[(size_t)j * r + i];
                sq = fmaf(v.x, v.x, fmaf(v.y, v.y, sq));
            }
            sq = warp_sum(sq);
            if (lane == 0) cn[j] = sq;
        }
        __syncthreads();
        int any = 0;
        float mo2 = 0.f;
        for (int base = 0; base < npair; base += nslots) {
            const int kp = base + slot;
            // round 0 of slot kp: (0, 1) for kp = 0, else (1 + kp, 1 + (rr - 1 - kp) % (rr - 1))
            int pa = kp == 0 ? 0 : 1 + kp;
            int pb = kp == 0 ? 1 : 1 + (rr - 1 - kp);
            if (pa > rr - 1) pa -= rr - 1;
            if (pb > rr - 1) pb -= rr - 1;
            for (int t = 0; t < rr - 1; ++t) {
                const int p = min(pa, pb), q = max(pa, pb);
                const bool valid = kp < npair && q < r && p != q;
                // a warp whose slots all lie beyond the round's pairs (r = 96: 48 pairs
                // for 64 slots) skips to the barrier instead of issuing the round on zeros
                // (up to r = 96; the longer columns leave no register for the test)
                if (EPL > 12 || base + (tid >> 5) * (32 / GL) < npair) {
                float2* cp = Rs + (size_t)p * r;
                float2* cq = Rs + (size_t)q * r;
                float2 x[EPL], y[EPL];
                if (V2) {
#pragma unroll
                    for (int v = 0; v < EPL / 2; ++v) {
                        const int i = 2 * (hl + GL * v);
                        float4 xv = make_float4(0.f, 0.f, 0.f, 0.f), yv = xv;
                        if (valid && i < r) {
                            xv = *(const float4*)(cp + i);
                            yv = *(const float4*)(cq + i);
                        }
                        x[2 * v] = make_float2(xv.x, xv.y);
                        x[2 * v + 1] = make_float2(xv.z, xv.w);
                        y[2 * v] = make_float2(yv.x, yv.y);
                        y[2 * v + 1] = make_float2(yv.z, yv.w);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < EPL; ++e) {
                        const int i = idx(e);
                        x[e] = y[e] = make_float2(0.f, 0.f);
                        if (valid && i < r) {
                            x[e] = cp[i];
                            y[e] = cq[i];
                        }
                    }
                }
                const float a = valid ? cn[p] : 0.f, b = valid ? cn[q] : 0.f;
                float2 g = make_float2(0.f, 0.f);
#pragma unroll
                for (int e = 0; e < EPL; ++e) cfmac(g, x[e], y[e]);
#pragma unroll
                for (int o = GL / 2; o > 0; o >>= 1) {
                    g.x += __shfl_xor_sync(0xffffffffu, g.x, o);
                    g.y += __shfl_xor_sync(0xffffffffu, g.y, o);
                }
                const float ag2 = fmaf(g.x, g.x, g.y * g.y), ab = a * b;
                if (valid && ab > 0.f) mo2 = fmaxf(mo2, __fdividef(ag2, ab));
                const bool rot = valid && a > 0.f && b > 0.f && ag2 >= 1.17549435e-38f && ag2 > tol2 * ab;
                if (rot) {
                    const float rg = rsqrt_nr(ag2);  // 1/|g|
                    const float2 ec = make_float2(g.x * rg, -g.y * rg);
                    const float zeta = (b - a) * 0.5f * rg;
                    const float tt = __fdividef(copysignf(1.f, zeta), fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
                    const float c = rsqrt_nr(fmaf(tt, tt, 1.f)), sn = c * tt;
                    if (hl == 0) {
                        const float tg = tt * (ag2 * rg);  // t |g|
                        cn[p] = fmaxf(a - tg, 0.f);
                        cn[q] = fmaxf(b + tg, 0.f);
                    }
                    float2 xn[EPL], yn[EPL];
#pragma unroll
                    for (int e = 0; e < EPL; ++e) {
                        const float2 ey = cmul(ec, y[e]);
                        xn[e] = make_float2(c * x[e].x - sn * ey.x, c * x[e].y - sn * ey.y);
                        yn[e] = make_float2(sn * x[e].x + c * ey.x, sn * x[e].y + c * ey.y);
                    }
                    if (V2) {
#pragma unroll
                        for (int v = 0; v < EPL / 2; ++v) {
                            const int i = 2 * (hl + GL * v);
                            if (i < r) {
                                *(float4*)(cp + i) = make_float4(xn[2 * v].x, xn[2 * v].y, xn[2 * v + 1].x,
                                                                 xn[2 * v + 1].y);
                                *(float4*)(cq + i) = make_float4(yn[2 * v].x, yn[2 * v].y, yn[2 * v + 1].x,
                                                                 yn[2 * v + 1].y);
                            }
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < EPL; ++e) {
                            const int i = idx(e);
                            if (i < r) {
                                cp[i] = xn[e];
                                cq[i] = yn[e];
                            }
                        }
                    }
                    for (int cc = hl; cc < np; cc += GL) {  // the rows p, q of d' (np right-hand sides)
                        const float2 xv = dp[p * np + cc];
                        const float2 ey = cmul(cconj(ec), dp[q * np + cc]);
                        dp[p * np + cc] = make_float2(c * xv.x - sn * ey.x, c * xv.y - sn * ey.y);
                        dp[q * np + cc] = make_float2(sn * xv.x + c * ey.x, sn * xv.y + c * ey.y);
                    }
                }
                any |= rot ? 1 : 0;
                }
                any = __syncthreads_or(any);
                // next round: both indices of a slot advance by one (kp = 0 keeps p = 0)
                if (kp != 0) pa = pa == rr - 1 ? 1 : pa + 1;
                pb = pb == rr - 1 ? 1 : pb + 1;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mo2 = fmaxf(mo2, __shfl_xor_sync(0xffffffffu, mo2, o));
        if (lane == 0) atomicMax(&max_off2, __float_as_int(mo2));
        __syncthreads();
        const float mo = __int_as_float(max_off2);
        __syncthreads();
        // no rotation, or the largest relative off-diagonal below sqrt(tol)
        if (!any || mo < tol) return sweep + 1;
    }
    return sweep;  // sweeps executed
}

template <typename T> struct JacobiSweeps {
    static __device__ int run(cplx<T>* Rs, cplx<T>* dp, int np, int r, int max_sweeps, T tol, T*) {
        return jacobi_sweeps_smem<T>(Rs, dp, np, r, max_sweeps, tol);
    }
};
template <> struct JacobiSweeps<float> {
    static __device__ int run(float2* Rs, float2* dp, int np, int r, int max_sweeps, float tol, float* cn) {
        const bool v2 = (r & 1) == 0;  // 16-byte pairs of entries need an even column length
        if (r <= 32) return v2 ? jacobi_sweeps_reg<4, true>(Rs, dp, np, r, max_sweeps, tol, cn)
                               : jacobi_sweeps_reg<4, false>(Rs, dp, np, r, max_sweeps, tol, cn);
        if (r <= 64) return v2 ? jacobi_sweeps_reg<8, true>(Rs, dp, np, r, max_sweeps, tol, cn)
                               : jacobi_sweeps_reg<8, false>(Rs, dp, np, r, max_sweeps, tol, cn);
        if (r <= 96) return v2 ? jacobi_sweeps_reg<12, true>(Rs, dp, np, r, max_sweeps, tol, cn)
                               : jacobi_sweeps_reg<12, false>(Rs, dp, np, r, max_sweeps, tol, cn);
        if (r <= 128) return v2 ? jacobi_sweeps_reg<16, true>(Rs, dp, np, r, max_sweeps, tol, cn)
                                : jacobi_sweeps_reg<16, false>(Rs, dp, np, r, max_sweeps, tol, cn);
        if (r <= 160) return v2 ? jacobi_sweeps_reg<20, true>(Rs, dp, np, r, max_sweeps, tol, cn)
                                : jacobi_sweeps_reg<20, false>(Rs, dp, np, r, max_sweeps, tol, cn);
        return jacobi_sweeps_smem<float>(Rs, dp, np, r, max_sweeps, tol);
    }
};

template <typename T>
__global__ void __launch_bounds__(JAC_THREADS)
k_jacobi(const cplx<T>* __restrict__ R, long ldr, long sR, const State* st, const cplx<T>* __restrict__ d, long sd,
         int np, T* sigma, long ssig, cplx<T>* UR, long ldu, long sU, cplx<T>* dprime, long sdp, int max_sweeps,
         int* sweeps_out, cplx<T>* gR, long sG) {
    // d and d' are r x np (np right-hand sides, row-major) per slice.  The
    // working copy of R (column-major) lives in shared memory, or, when gR is
    // given (factors too large for shared memory: the full T-tSVD), in gR +
    // s sG in global memory (the slices' copies stay in L2).
    typedef cplx<T> V;
    const int r = st->r;
    if (r <= 0) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* Rs = gR ? gR + (long)blockIdx.x * sG : (V*)smraw;  // column j at Rs[j*r]
    V* dp = gR ? (V*)smraw : Rs + (size_t)r * r;
    T* sg = (T*)(dp + (size_t)r * np);  // column norms (sigma), working precision
    int* perm = (int*)(sg + r);
    __shared__ T tol_s;
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    R += (long)s * sR;
    for (int e = tid; e < r * r; e += blockDim.x) {
        const int i = e / r, j = e - i * r;
        Rs[(size_t)j * r + i] = R[(long)i * ldr + j];
    }
    for (int i = tid; i < r * np; i += blockDim.x) dp[i] = d[(long)s * sd + i];
    if (tid == 0) tol_s = (T)(4.0 * sqrt((double)r) * Eps<T>::v);
    __syncthreads();
    const int sweep = JacobiSweeps<T>::run(Rs, dp, np, r, max_sweeps, tol_s, sg);  // sg: the sweeps' norm scratch
    for (int j = warp; j < r; j += nw) {
        T a = 0;  // column norms in the working precision (float64 only on lane 0)
        for (int i = lane; i < r; i += 32) a += cabs2(Rs[(size_t)j * r + i]);
        a = warp_sum(a);
        if (lane == 0) sg[j] = sqrt(a);
    }
    __syncthreads();
    for (int j = tid; j < r; j += blockDim.x) {
        int rank = 0;
        const T v = sg[j];
        for (int i = 0; i < r; ++i) rank += (sg[i] > v) || (sg[i] == v && i < j);
        perm[rank] = j;
    }
    __syncthreads();
    for (int e = tid; e < r * np; e += blockDim.x) {
        const int jr = e / np, cc = e - jr * np;
        const int j = perm[jr];
        if (cc == 0) sigma[(long)s * ssig + jr] = sg[j];
        dprime[(long)s * sdp + e] = dp[j * np + cc];
    }
    V* U = UR + (long)s * sU;
    for (int e = tid; e < r * r; e += blockDim.x) {
        const int i = e / r, jr = e - i * r;
        const int j = perm[jr];
        const T sv = sg[j];
        const V x = Rs[(size_t)j * r + i];
        U[(long)i * ldu + jr] = sv > (T)0 ? cscale(x, (T)1 / sv) : mk<T>(0, 0);
    }
    if (tid == 0) atomicMax(sweeps_out, sweep);
}

static size_t jacobi_smem(int r, size_t c, int np, bool global_r = false) {
    return (global_r ? 0 : (size_t)r * r * c) + (size_t)r * np * c + (size_t)r * sizeof(double) +
           (size_t)r * sizeof(int);
}

// The one-sided Jacobi SVD of h square r x r factors (r from st->r, at most
// r_max), with np right-hand sides rotated along; see k_jacobi.
template <typename T>
tp_status jacobi_svd(int h, const void* R, long ldr, long sR, const State* st, const void* d, long sd, int np,
                     T* sigma, long ssig, void* UR, long ldu, long sU, void* dprime, long sdp, int r_max,
                     int* sweeps, cudaStream_t stream) {
    const size_t smem = jacobi_smem(r_max, sizeof(cplx<T>), np);
    if (smem > 227 * 1024) return TP_ERR_UNSUPPORTED;
    if (smem_optin((const void*)k_jacobi<T>, smem) != TP_OK) return TP_ERR_CUDA;
    prof_begin(TP_KC_SVD, stream);
    k_jacobi<T><<<h, JAC_THREADS, smem, stream>>>((const cplx<T>*)R, ldr, sR, st, (const cplx<T>*)d, sd, np, sigma,
                                                  ssig, (cplx<T>*)UR, ldu, sU, (cplx<T>*)dprime, sdp, 60, sweeps,
                                                  nullptr, 0);
    return launched(TP_KC_SVD, stream);
}
template tp_status jacobi_svd<float>(int, const void*, long, long, const State*, const void*, long, int, float*, long,
                                     void*, long, long, void*, long, int, int*, cudaStream_t);
template tp_status jacobi_svd<double>(int, const void*, long, long, const State*, const void*, long, int, double*,
                                      long, void*, long, long, void*, long, int, int*, cudaStream_t);

// alpha_j = d'_j / sigma_j^pw (pw = 1: the solution coefficients; pw = 2:
// the adjoint's), dropping sigma_j <= dims * eps * sigma_max.
template <typename T>
__global__ void k_alpha(const T* sigma, long ssig, const cplx<T>* dprime, long sdp, cplx<T>* alpha, long sa,
                        const State* st, int h, int dims, int r_max, int np, int pw = 1) {
    __shared__ double red[32];
    const int r = st->r, s = blockIdx.x;
    double mx = 0.0;
    for (int i = threadIdx.x; i < h; i += blockDim.x) mx = fmax(mx, (double)sigma[(long)i * ssig]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    double gmax = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) gmax = fmax(gmax, red[w]);
    const double tol = (double)dims * Eps<T>::v * gmax;
    for (int e = threadIdx.x; e < r_max * np; e += blockDim.x) {  // alpha, d' are r_max x np
        const int j = e / np;
        cplx<T> a = mk<T>(0, 0);
        if (j < r) {
            const double sv = (double)sigma[(long)s * ssig + j];
            if (sv > tol) {
                const cplx<T> v = dprime[(long)s * sdp + e];
                const double dv = pw == 2 ? sv * sv : sv;
                a = mk<T>((T)(v.x / dv), (T)(v.y / dv));
            }
        }
        alpha[(long)s * sa + e] = a;
    }
}

// Coefficients in the computed basis.  The one-sided Jacobi stops when every
// pair of columns of R J is orthogonal to within its tolerance (relative
// off-diagonal 4 sqrt(r) u), so the normalised columns U_R are orthonormal only
// to that level, and the sum of alpha_j v_j over j < k with alpha_j = d'_j /
// sigma_j treats U_k^H U_k as the identity.  For the truncated solution in the
// span of V_k = Q_G U_k the coefficients are (U_k^H U_k)^{-1} alpha_k; with
// N = U_k^H U_k - I of order 1e-6 its first-order form
//   alpha_k <- alpha_k - N alpha_k = 2 alpha_k - U_k^H (U_k alpha_k)
// is exact to O(|N|^2).  In float32 this takes the error of the 256^3
// truncated solution from 1.8e-5 to 1e-6 against the float64 oracle.  k from
// the state (the discrepancy choice), r the sketch rank; alpha is r_max x np
// per slice (row-major), U_R row-major with column j the j-th singular vector.
// Applied in the same way to t = V_k^H G of the adjoint (the map is
// self-adjoint in the coefficients).  Right-hand sides in chunks of 16.
template <typename T>
__global__ void __launch_bounds__(256) k_alpha_corr(const cplx<T>* __restrict__ UR, long ldu, long sU,
                                                   cplx<T>* alpha, long sa, const State* st, int np) {
    typedef cplx<T> V;
    constexpr int CH = 16;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int r = st->r, k = st->k, s = blockIdx.x;
    if (k <= 0 || r <= 0) return;
    V* a = (V*)smraw;      // k x nc: the coefficients of this chunk
    V* t = a + k * CH;     // r x nc: U_k a
    const V* U = UR + (long)s * sU;
    V* al = alpha + (long)s * sa;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int c0 = 0; c0 < np; c0 += CH) {
        const int nc = np - c0 < CH ? np - c0 : CH;
        for (int e = tid; e < k * nc; e += blockDim.x) {
            const int j = e / nc, c = e - j * nc;
            a[e] = al[(long)j * np + c0 + c];
        }
        __syncthreads();
        // t_i = sum_{j<k} U[i][j] a_j: a warp per (row, column), lanes along the row
        for (int ic = warp; ic < r * nc; ic += nw) {
            const int i = ic / nc, c = ic - i * nc;
            V acc = mk<T>(0, 0);
            for (int j = lane; j < k; j += 32) cfma(acc, U[(long)i * ldu + j], a[j * nc + c]);
            acc.x = warp_sum(acc.x);
            acc.y = warp_sum(acc.y);
            if (lane == 0) t[i * nc + c] = acc;
        }
        __syncthreads();
        // alpha_j <- 2 a_j - sum_i conj(U[i][j]) t_i: a thread per (j, column), consecutive threads along j
        for (int e = tid; e < k * nc; e += blockDim.x) {
            const int c = e / k, j = e - c * k;
            V acc = mk<T>(0, 0);
            for (int i = 0; i < r; ++i) cfmac(acc, U[(long)i * ldu + j], t[i * nc + c]);
            const V x = a[j * nc + c];
            al[(long)j * np + c0 + c] = mk<T>((T)2 * x.x - acc.x, (T)2 * x.y - acc.y);
        }
        __syncthreads();
    }
}

template <typename T>
static tp_status alpha_corr(int h, const cplx<T>* UR, int r_max, cplx<T>* alpha, long sa, const State* st, int np,
                            cudaStream_t stream) {
    const size_t smem = (size_t)2 * r_max * 16 * sizeof(cplx<T>);
    if (smem_optin((const void*)k_alpha_corr<T>, smem) != TP_OK) return TP_ERR_CUDA;
    prof_begin(TP_KC_MISC, stream);
    k_alpha_corr<T><<<h, 256, smem, stream>>>(UR, r_max, (long)r_max * r_max, alpha, sa, st, np);
    return launched(TP_KC_MISC, stream);
}

// Per slice: squared residual norms ||b - sum_{j<k} K_j alpha^(k)_j||^2 for
// the candidates k = k_init .. r (k_init = max(1, r - p), Eq. (kinit)), where
// K = A V (stored vector-major, K_j contiguous) and alpha^(k) are the
// coefficients that the solution truncated at k uses: in float32 the
// computed-basis coefficients 2 alpha_k - U_k^H (U_k alpha_k) of
// k_alpha_corr (so that the residual tested is the returned solution's), in
// float64 alpha_k itself (U_R orthonormal to rounding).  Up to DP_CC
// candidates share one pass over K: each thread carries its RPT rows of every
// candidate's residual.  np right-hand sides (alpha and B row-major with np
// columns): a CTA per (slice, column, candidate group), column c writing its
// squared norms to out + c h so (the reduction sums the columns); the
// candidates are split evenly over gridDim.z CTAs, each writing its own
// entries (the first also the zeros).  Per thread and per warp in the working
// precision, across warps in float64.
constexpr int DP_CC = 12;
template <typename T, int RPT>
__global__ void __launch_bounds__(256)
k_dp_scan(const cplx<T>* __restrict__ KhT, long sK, const cplx<T>* __restrict__ alpha, long sa,
          const cplx<T>* __restrict__ bhat, long sb, const cplx<T>* __restrict__ UR, long ldu, long sU,
          const State* st, int l, int np, int p_over, double* out, long so) {
    typedef cplx<T> V;
    constexpr bool CORR = sizeof(T) == 4;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int r = st->r, s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = blockDim.x >> 5, c = blockIdx.y;
    out += (long)c * gridDim.x * so;
    double* wsum = (double*)smraw;                        // [nw][r+1]
    V* Tm = (V*)(wsum + (size_t)nw * (r + 1) + 1);        // r x DP_CC: U_k alpha_k per candidate
    V* ak = Tm + (size_t)r * DP_CC;                       // DP_CC x r: alpha^(k), zero for j >= k
    Tm = (V*)(((size_t)Tm + 15) & ~(size_t)15);
    ak = Tm + (size_t)r * DP_CC;
    const int k_init = max(1, r - p_over), ncand = r - k_init + 1;
    const int per = (ncand + gridDim.z - 1) / gridDim.z;
    const int q_lo = blockIdx.z * per, q_hi = min(ncand, q_lo + per);  // this CTA's candidates k_init + q
    KhT += (long)s * sK;
    const V* al = alpha + (long)s * sa;
    const V* U = UR + (long)s * sU;
    for (int e = tid; e < nw * (r + 1); e += blockDim.x) wsum[e] = 0.0;
    {
        for (int c0 = q_lo; c0 < q_hi; c0 += DP_CC) {
            const int nc = min(DP_CC, q_hi - c0), kb = k_init + c0;  // candidates kb .. kb + nc - 1
            if (CORR) {
                // T[i][q] = sum_{j < kb+q} U[i][j] a_j: the first column in full, the others by one more
                // term each (a thread per row i)
                for (int i = tid; i < r; i += blockDim.x) {
                    V acc = mk<T>(0, 0);
                    const V* Ui = U + (long)i * ldu;
#pragma unroll 4
                    for (int j = 0; j < kb; ++j) cfma(acc, Ui[j], al[(long)j * np + c]);
                    Tm[i * DP_CC] = acc;
                    for (int q = 1; q < nc; ++q) {
                        const int j = kb + q - 1;
                        cfma(acc, Ui[j], al[(long)j * np + c]);
                        Tm[i * DP_CC + q] = acc;
                    }
                }
                __syncthreads();
                // alpha^(k)_j = 2 a_j - sum_i conj(U[i][j]) T[i][q]
                for (int e = tid; e < r * nc; e += blockDim.x) {
                    const int q = e / r, j = e - q * r;
                    V v = mk<T>(0, 0);
                    if (j < kb + q) {
                        V acc = mk<T>(0, 0);
#pragma unroll 4
                        for (int i = 0; i < r; ++i) cfmac(acc, U[(long)i * ldu + j], Tm[i * DP_CC + q]);
                        const V a = al[(long)j * np + c];
                        v = mk<T>((T)2 * a.x - acc.x, (T)2 * a.y - acc.y);
                    }
                    ak[q * r + j] = v;
                }
            } else {
                for (int e = tid; e < r * nc; e += blockDim.x) {
                    const int q = e / r, j = e - q * r;
                    ak[q * r + j] = j < kb + q ? al[(long)j * np + c] : mk<T>(0, 0);
                }
            }
            __syncthreads();
            V res[DP_CC][RPT];
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                const int i = tid + u * blockDim.x;
                const V b = (i < l) ? bhat[(long)s * sb + (long)i * np + c] : mk<T>(0, 0);
#pragma unroll
                for (int q = 0; q < DP_CC; ++q) res[q][u] = b;
            }
            // the K loads of the next DP_PF columns are in flight while one is applied
            constexpr int DP_PF = (8 * 4 / (int)sizeof(T)) / RPT > 2 ? (8 * 4 / (int)sizeof(T)) / RPT : 2;
            const int kend = kb + nc - 1;
            V kv[DP_PF][RPT];
#pragma unroll
            for (int f = 0; f < DP_PF; ++f)
#pragma unroll
                for (int u = 0; u < RPT; ++u) {
                    const int i = tid + u * blockDim.x;
                    kv[f][u] = (i < l && f < kend) ? KhT[(long)f * l + i] : mk<T>(0, 0);
                }
            for (int j0 = 0; j0 < kend; j0 += DP_PF) {
#pragma unroll
                for (int f = 0; f < DP_PF; ++f) {
                    const int j = j0 + f;
                    if (j >= kend) break;
                    V cur[RPT];
#pragma unroll
                    for (int u = 0; u < RPT; ++u) {
                        cur[u] = kv[f][u];
                        const int i = tid + u * blockDim.x;
                        const int jn = j + DP_PF;
                        kv[f][u] = (i < l && jn < kend) ? KhT[(long)jn * l + i] : mk<T>(0, 0);
                    }
#pragma unroll
                    for (int q = 0; q < DP_CC; ++q) {
                        if (q >= nc) break;
                        const V a = ak[q * r + j];
#pragma unroll
                        for (int u = 0; u < RPT; ++u) res[q][u] = csub(res[q][u], cmul(cur[u], a));
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < DP_CC; ++q) {
                if (q >= nc) break;
                T part = 0;
#pragma unroll
                for (int u = 0; u < RPT; ++u) part += cabs2(res[q][u]);
                part = warp_sum(part);
                if (lane == 0) wsum[warp * (r + 1) + kb + q] += (double)part;
            }
            __syncthreads();
        }
    }
    for (int j = tid; j <= r; j += blockDim.x) {
        const int q = j - k_init;
        const bool mine = q >= q_lo && q < q_hi;
        if (!mine && !(blockIdx.z == 0 && q < 0)) continue;  // other CTAs' candidates
        double a = 0.0;
        if (mine)
            for (int w = 0; w < nw; ++w) a += wsum[w * (r + 1) + j];
        out[(long)s * so + j] = a;
    }
}

template <typename T>
static tp_status dp_scan(int h, const cplx<T>* KhT, long sK, const cplx<T>* alpha, long sa, const cplx<T>* bhat,
                         long sb, const cplx<T>* UR, int r_max, const State* st, int l, int np, int p_over,
                         double* out, long so, cudaStream_t stream) {
    const size_t smem = (size_t)8 * (r_max + 1) * sizeof(double) + 16 + 2 * (size_t)r_max * DP_CC * sizeof(cplx<T>);
    auto kern = l <= 256 ? k_dp_scan<T, 1> : (l <= 512 ? k_dp_scan<T, 2> : k_dp_scan<T, 4>);
    if (smem_optin((const void*)kern, smem) != TP_OK) return TP_ERR_CUDA;
    prof_begin(TP_KC_DP, stream);
    // the candidates k_init..r (at most p + 1) over up to four CTAs per slice and column
    const int nz = std::min(4, std::max(1, (std::min(p_over, r_max - 1) + 1 + 3) / 4));
    kern<<<dim3((unsigned)h, (unsigned)np, (unsigned)nz), 256, smem, stream>>>(
        KhT, sK, alpha, sa, bhat, sb, UR, r_max, (long)r_max * r_max, st, l, np, p_over, out, so);
    return launched(TP_KC_DP, stream);
}

// Global residuals (Parseval over slices), the discrepancy-principle choice
// of k in [max(1, r-p), r], and the info record.
__global__ void k_dp_reduce(const double* out, long so, int h, int np, int n, State* st, int p_over,
                            double tau_delta, tp_info* info, double* res_hist, int r_max) {
    extern __shared__ double res[];
    const int r = st->r;
    const int k_init = max(1, r - p_over);  // only the candidates k_init..r are needed
    // one warp per candidate k: lanes take every 32nd slice (their loads all
    // in flight), then a fixed-order warp sum
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = k_init + warp; k <= r; k += nw) {
        double a = 0.0;
        for (int c = 0; c < np; ++c)  // the right-hand sides' partials, in a fixed order
            for (int s = lane; s < h; s += 32) a += parseval_w(s, n) * out[((long)c * h + s) * so + k];
        a = warp_sum(a);
        if (lane == 0) res[k] = sqrt(fmax(a, 0.0) / (double)n);
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    int k = r, status = TP_ERR_NOT_CONVERGED;
    for (int j = k_init; j <= r; ++j)
        if (res[j] <= tau_delta) {
            k = j;
            status = TP_OK;
            break;
        }
    if (st->eps2 >= 0.0 && st->eta >= st->eps2) status = TP_ERR_NOT_CONVERGED;
    if (st->status == TP_ERR_TIMEOUT) status = TP_ERR_TIMEOUT;  // a bounded wait of a product ran out
    if (st->nonfinite) status = TP_ERR_NONFINITE;
    double margin = fabs(res[k] - tau_delta) / tau_delta;
    if (k - 1 >= k_init) margin = fmin(margin, fabs(res[k - 1] - tau_delta) / tau_delta);
    st->k = k;
    st->status = status;
    if (res_hist)
        for (int j = 0; j <= r_max; ++j) res_hist[j] = (j >= k_init && j <= r) ? res[j] : -1.0;
    tp_info o;
    o.status = status;
    o.k = k;
    o.r = r;
    o.sweeps = st->sweeps;
    o.residual = st->nonfinite ? __longlong_as_double(0x7ff8000000000000LL) : res[k];  // NaN
    o.tau_delta = tau_delta;
    o.eta = st->eta;
    o.mu = 0.0;
    o.margin = margin;
    o.norm_a2 = st->norm_a2;
    *info = o;
}

// ---------------------------------------------------------------------------
// Workspace layout and the solve.
// ---------------------------------------------------------------------------
template <typename T>
struct RtWs {
    State* st;
    double *partsA, *partsB, *normsq, *dpout;
    cplx<T> *Ahat, *AhT, *Bhat, *G, *Y, *Z, *Q, *BHb, *QG, *R, *d, *UR, *dprime, *alpha, *Vt, *KhT, *Xhat;
    T* sigma;
    __nv_bfloat162 *Abf, *ATbf;
    size_t bytes;
};

// A-hat^T per slice (m x l), so that the float32 products A-hat^H Y read rows
// (conj(A-hat^T) Y) on the tensor cores.  32 x 32 tiles through shared memory.
// In the BF16 form (Abf, ATbf not null) the same pass also writes bfloat16
// copies of A-hat and A-hat^T (re, im rounded to nearest, 4 bytes per entry).
template <typename T>
__global__ void __launch_bounds__(256) k_ctranspose(const cplx<T>* __restrict__ A, cplx<T>* __restrict__ AT, int l,
                                                    int m, __nv_bfloat162* Abf, __nv_bfloat162* ATbf) {
    __shared__ cplx<T> tile[32][33];
    const long s = blockIdx.z;
    const int j0 = blockIdx.x * 32, i0 = blockIdx.y * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    A += s * l * m;
    AT += s * l * m;
    for (int y = ty; y < 32; y += 8) {
        const int i = i0 + y, j = j0 + tx;
        if (i < l && j < m) {
            const cplx<T> v = A[(long)i * m + j];
            tile[y][tx] = v;
            if (Abf) Abf[s * l * m + (long)i * m + j] = __floats2bfloat162_rn((float)v.x, (float)v.y);
        }
    }
    __syncthreads();
    for (int y = ty; y < 32; y += 8) {
        const int j = j0 + y, i = i0 + tx;
        if (i < l && j < m) {
            const cplx<T> v = tile[tx][y];
            AT[(long)j * l + i] = v;
            if (ATbf) ATbf[s * l * m + (long)j * l + i] = __floats2bfloat162_rn((float)v.x, (float)v.y);
        }
    }
}

template <typename T>
static RtWs<T> rt_carve(void* base, int l, int m, int n, int b, int r_max, int p, bool bf16 = false) {
    typedef cplx<T> V;
    const long h = n / 2 + 1;
    Carver c(base, 0);
    RtWs<T> w;
    w.st = c.take<State>(1);
    w.partsA = c.take<double>(rdft_parts(l, m));
    w.partsB = c.take<double>(rdft_parts(l, p));
    w.normsq = c.take<double>(h);
    w.dpout = c.take<double>(h * (r_max + 1) * p);  // per right-hand side
    w.Ahat = c.take<V>(h * l * m);
    w.AhT = sizeof(T) == 4 ? c.take<V>(h * l * m) : nullptr;  // float32 only: tensor-core products
    w.Bhat = c.take<V>(h * l * p);
    w.G = c.take<V>(h * m * r_max);  // all Gaussian slices, transformed once
    w.Y = c.take<V>(h * l * b);
    w.Z = c.take<V>(h * m * b);
    w.Q = c.take<V>(h * r_max * l);
    w.BHb = c.take<V>(h * m * b);
    w.QG = c.take<V>(h * r_max * m);
    w.R = c.take<V>(h * r_max * r_max);
    w.d = c.take<V>(h * r_max * p);
    w.UR = c.take<V>(h * r_max * r_max);
    w.dprime = c.take<V>(h * r_max * p);
    w.alpha = c.take<V>(h * r_max * p);
    w.Vt = c.take<V>(h * m * r_max);
    w.KhT = c.take<V>(h * r_max * l);
    w.Xhat = c.take<V>(h * m * p);
    w.sigma = c.take<T>(h * r_max);
    // BF16 form only, after everything else (the other layouts do not move):
    // bfloat16 copies of A-hat and A-hat^T for the sketch and power products
    w.Abf = bf16 ? c.take<__nv_bfloat162>(h * l * m) : nullptr;
    w.ATbf = bf16 ? c.take<__nv_bfloat162>(h * l * m) : nullptr;
    w.bytes = c.off;
    return w;
}

static int jac_rmax(size_t elem, int p) {
    // largest r whose Jacobi working set (p right-hand sides) fits in 227 KB of shared memory
    int r = 1;
    while (jacobi_smem(r + 1, 2 * elem, p) <= 227 * 1024) ++r;
    return r;
}

constexpr int RT_MAX_RHS = 64;    // lateral slices of B per RT-tSVD call
constexpr int RT_MAX_RANK = 256;  // sketch rank (the small SVD of rank above jac_rmax runs from global memory)

template <typename T>
static tp_status rt_check(int l, int m, int n, int p, const tp_rtsvd_params* P, bool full = false) {
    if (!P || l < 1 || m < 1 || n < 1 || p < 1 || p > RT_MAX_RHS) return TP_ERR_ARG;
    if (l > 1024 || m > 1024 || n > (sizeof(T) == 4 ? 1024 : 512)) return TP_ERR_ARG;
    if (P->block < 1 || P->block > MAX_BLOCK || P->r_max < 1 || P->r_max > (l < m ? l : m)) return TP_ERR_ARG;
    // the small SVD: in shared memory up to jac_rmax, beyond it (up to 256) with R's working copy in global
    // memory and only the p right-hand sides in shared memory
    if (P->r_max > RT_MAX_RANK) return TP_ERR_ARG;
    if (P->r_max > jac_rmax(sizeof(T), p) && jacobi_smem(P->r_max, 2 * sizeof(T), p, true) > 227 * 1024)
        return TP_ERR_ARG;
    if (!(P->tau > 0.0) || !(P->delta >= 0.0) || P->p_over < 0 || P->q_power < 0) return TP_ERR_ARG;
    if (!full && !(P->eps > 0.0) && !(P->eps_rel > 0.0)) return TP_ERR_ARG;
    const int Lmax = l > m ? l : m;
    if (orth_smem(Lmax, P->block, P->r_max, 2 * sizeof(T)) > 227 * 1024) return TP_ERR_ARG;
    return TP_OK;
}

template <typename T>
size_t rt_ws_bytes(int l, int m, int n, int p, const tp_rtsvd_params* P, bool bf16) {
    if (rt_check<T>(l, m, n, p, P) != TP_OK) return 0;
    if (bf16 && sizeof(T) != 4) return 0;
    return rt_carve<T>(nullptr, l, m, n, P->block, P->r_max, p, bf16).bytes;
}

#define TRY(x)                              \
    do {                                    \
        tp_status _e = (x);                 \
        if (_e != TP_OK) return _e;         \
    } while (0)

template <typename T>
static tp_status rt_solve_impl(const T* A, const T* B, const T* Om, int l, int m, int n, int p,
                               const tp_rtsvd_params* P, T* X, tp_info* info, void* ws, size_t ws_bytes,
                               cudaStream_t st, int tc_passes, bool full, const void* Ahat_in = nullptr) {
    TRY(rt_check<T>(l, m, n, p, P, full));
    if ((!A && !Ahat_in) || !B || !Om || !X || !info) return TP_ERR_ARG;
    if (Ahat_in && ((size_t)Ahat_in & 15)) return TP_ERR_ARG;
    const int b = P->block, r_max = P->r_max, h = n / 2 + 1;
    // tc_passes: 3 = float32-accurate products, 1 = the TF32 form, 0 = the BF16
    // form (sketch and power products on bfloat16 copies of A-hat)
    const bool bf16 = tc_passes == 0;
    // the bfloat16 products read 16-byte multiples per row (4 complex entries): refused before anything runs
    if (bf16 && (sizeof(T) != 4 || (l & 3) || (m & 3))) return TP_ERR_ARG;
    RtWs<T> w = rt_carve<T>(ws, l, m, n, b, r_max, p, bf16);
    if (!ws || ((size_t)ws & 255) || ws_bytes < w.bytes) return TP_ERR_WORKSPACE;
    const long lm = (long)l * m;
    const int* done = &w.st->done;

    if (Ahat_in) {  // the caller's half spectrum of A (read only); ||A||^2 by Parseval
        w.Ahat = (cplx<T>*)Ahat_in;
        TRY(norm2_hat<T>(Ahat_in, n, l, m, w.partsA, st));
    } else {
        TRY(rdft<T>(A, w.Ahat, n, l, m, m, lm, w.partsA, nullptr, st));
    }
    if (w.AhT) {
        prof_begin(TP_KC_GEMM, st);
        k_ctranspose<T><<<dim3((unsigned)((m + 31) / 32), (unsigned)((l + 31) / 32), (unsigned)h), 256, 0, st>>>(
            w.Ahat, w.AhT, l, m, w.Abf, w.ATbf);
        TRY(launched(TP_KC_GEMM, st));
    }
    // A-hat^H Y: conj(A-hat^T) Y from the transposed copy when there is one
    const cplx<T>* AH = w.AhT ? w.AhT : w.Ahat;
    const long ldah = w.AhT ? l : m;
    const int op_h = w.AhT ? OP_R : OP_C;
    TRY(rdft<T>(B, w.Bhat, n, l, p, p, (long)l * p, w.partsB, nullptr, st));
    prof_begin(TP_KC_MISC, st);
    k_rt_init<<<1, 256, 0, st>>>(w.st, w.partsA, rdft_parts(l, m), w.partsB, rdft_parts(l, p), P->eps, P->eps_rel, n);
    TRY(launched(TP_KC_MISC, st));

    // all Gaussian slices -> Fourier in one launch (blocks the sketch never
    // reaches are transformed too; one full launch beats a latency-bound
    // launch per block)
    TRY(rdft<T>(Om, w.G, n, m, r_max, r_max, (long)m * r_max, nullptr, nullptr, st));
    // the sketch and power-iteration products: A-hat (op N) or conj(A-hat^T) (op R); in the BF16 form on the
    // bfloat16 copies, tensor cores only (a shape they do not take is refused, never run on other data)
    auto sketch = [&](int M, int N, int K, const void* Af, const void* Ab, long lda, int op, const cplx<T>* Bm,
                      long ldb, long sB, cplx<T>* C, long ldc, long sC) -> tp_status {
        if (!bf16)
            return cgemm<T>(h, M, N, K, 0, 0, 0, 1, 0, Af, lda, lm, op, Bm, ldb, sB, OP_N, 0, 0, C, ldc, sC, done, st,
                            &w.st->status, tc_passes);
        // a right-hand side that does not start on a 16-byte boundary (the columns of an odd block of Omega)
        // cannot be a TMA source: that product runs float32-accurate on the float32 A-hat instead
        if (((uintptr_t)Bm & 15) || (ldb & 1) || (sB & 1))
            return cgemm<T>(h, M, N, K, 0, 0, 0, 1, 0, Af, lda, lm, op, Bm, ldb, sB, OP_N, 0, 0, C, ldc, sC, done,
                            st, &w.st->status, 3);
        const tp_status e = zgemm_tc(h, M, N, K, Ab, lda, lm, op, Bm, ldb, sB, C, ldc, sC, done, &w.st->status, 0,
                                     st);
        return e == TP_ERR_UNSUPPORTED ? TP_ERR_ARG : e;
    };
    const int nblk = (r_max + b - 1) / b;
    for (int blk = 0; blk < nblk; ++blk) {
        const int r0 = blk * b, bb = (b < r_max - r0) ? b : r_max - r0;
        // sketch, power iterations, orthonormalise
        TRY(sketch(l, bb, m, w.Ahat, w.Abf, m, OP_N, w.G + r0, r_max, (long)m * r_max, w.Y, bb, (long)l * bb));
        const bool last_y = (P->q_power == 0);
        TRY(orth<T>(h, w.Y, (long)l * bb, l, bb, w.Q, (long)r_max * l, r0, last_y ? w.Q : nullptr, nullptr, 0, 0, 0,
                    nullptr, done, st));
        for (int it = 0; it < P->q_power; ++it) {
            TRY(sketch(m, bb, l, AH, w.ATbf, ldah, op_h, w.Y, bb, (long)l * bb, w.Z, bb, (long)m * bb));
            TRY(orth<T>(h, w.Z, (long)m * bb, m, bb, nullptr, 0, 0, nullptr, nullptr, 0, 0, 0, nullptr, done, st));
            TRY(sketch(l, bb, m, w.Ahat, w.Abf, m, OP_N, w.Z, bb, (long)m * bb, w.Y, bb, (long)l * bb));
            const bool last = (it + 1 == P->q_power);
            TRY(orth<T>(h, w.Y, (long)l * bb, l, bb, w.Q, (long)r_max * l, r0, last ? w.Q : nullptr, nullptr, 0, 0,
                        0, nullptr, done, st));
        }
        // Bt(block)^H = A^H Y; its QR against the earlier columns extends QG and R
        TRY(cgemm<T>(h, m, bb, l, 0, 0, 0, 1, 0, AH, ldah, lm, op_h, w.Y, bb, (long)l * bb, OP_N, 0, 0, w.BHb, bb,
                     (long)m * bb, done, st, &w.st->status, 3));  // the re-projection stays float32-accurate
        // its last CTA also takes the block's eta update
        TRY(orth<T>(h, w.BHb, (long)m * bb, m, bb, w.QG, (long)r_max * m, r0, w.QG, w.R, r_max,
                    (long)r_max * r_max, r_max, w.normsq, done, st, w.st, n, r0 + bb));
    }
    const int* dr = &w.st->r;
    // d = Q^H B (r_max x p per slice)
    const long rp = (long)r_max * p;
    TRY(cgemm<T>(h, r_max, p, l, dr, 0, 0, 1, 0, w.Q, l, (long)r_max * l, OP_R, w.Bhat, p, (long)l * p, OP_N, 0, 0,
                 w.d, p, rp, nullptr, st));
    {
        // factors too large for shared memory: the working copy in Vt (free until V = Q_G U_R is formed)
        const bool gmode = r_max > jac_rmax(sizeof(T), p);
        const size_t smem = jacobi_smem(r_max, sizeof(cplx<T>), p, gmode);
        if (smem_optin((const void*)k_jacobi<T>, smem) != TP_OK) return TP_ERR_CUDA;
        prof_begin(TP_KC_SVD, st);
        k_jacobi<T><<<h, JAC_THREADS, smem, st>>>(w.R, r_max, (long)r_max * r_max, w.st, w.d, rp, p, w.sigma, r_max,
                                                    w.UR, r_max, (long)r_max * r_max, w.dprime, rp, 60,
                                                    &w.st->sweeps, gmode ? w.Vt : nullptr, (long)m * r_max);
        TRY(launched(TP_KC_SVD, st));
    }
    prof_begin(TP_KC_MISC, st);
    k_alpha<T><<<h, 256, 0, st>>>(w.sigma, r_max, w.dprime, rp, w.alpha, rp, w.st, h, l > m ? l : m, r_max, p);
    TRY(launched(TP_KC_MISC, st));
    // V = QG^T-as-matrix * U_R ;  K^T = V^T A^T (vector-major K = A V)
    TRY(cgemm<T>(h, m, r_max, r_max, 0, dr, dr, 1, 0, w.QG, m, (long)r_max * m, OP_T, w.UR, r_max,
                 (long)r_max * r_max, OP_N, 0, 0, w.Vt, r_max, (long)m * r_max, nullptr, st));
    // float32: K = A-hat V on the tensor cores in column chunks of 32, written
    // transposed; chunks past the sketch rank r are skipped on the device
    bool k_done = false;
    if (sizeof(T) == 4) {
        tp_status e = TP_OK;
        for (int c0 = 0; c0 < r_max && e == TP_OK; c0 += 32) {
            const int nc = r_max - c0 < 32 ? r_max - c0 : 32;
            e = zgemm_tc(h, l, nc, m, w.Ahat, m, lm, OP_N, w.Vt + c0, r_max, (long)m * r_max, w.KhT + (long)c0 * l,
                         l, (long)r_max * l, nullptr, &w.st->status, 3, st, 1, dr, c0);
            if (c0 == 0 && e == TP_ERR_UNSUPPORTED) break;  // shape not taken: the SIMT product below
            TRY(e);
            k_done = e == TP_OK;
        }
    }
    if (!k_done)
        TRY(cgemm<T>(h, r_max, l, m, dr, 0, 0, 1, 0, w.Vt, r_max, (long)m * r_max, OP_T, w.Ahat, m, lm, OP_T, 0, 0,
                     w.KhT, l, (long)r_max * l, nullptr, st));
    TRY(dp_scan<T>(h, w.KhT, (long)r_max * l, w.alpha, rp, w.Bhat, (long)l * p, w.UR, r_max, w.st, l, p, P->p_over,
                   w.dpout, r_max + 1, st));
    prof_begin(TP_KC_DP, st);
    k_dp_reduce<<<1, 256, (r_max + 1) * sizeof(double), st>>>(w.dpout, r_max + 1, h, p, n, w.st, P->p_over,
                                                              P->tau * P->delta, info, P->res_hist, r_max);
    TRY(launched(TP_KC_DP, st));
    // float32: the coefficients of the chosen k in the computed (not exactly orthonormal) basis
    if (sizeof(T) == 4) TRY(alpha_corr<T>(h, w.UR, r_max, w.alpha, rp, w.st, p, st));
    TRY(cgemm<T>(h, m, p, r_max, 0, 0, &w.st->k, 1, 0, w.Vt, r_max, (long)m * r_max, OP_N, w.alpha, p, rp, OP_N,
                 0, 0, w.Xhat, p, (long)m * p, nullptr, st));
    TRY(irdft<T>(w.Xhat, X, n, m, p, p, (long)m * p, nullptr, st));
    return TP_OK;
}

template <typename T>
tp_status rt_solve(const T* A, const T* B, const T* Om, int l, int m, int n, int p, const tp_rtsvd_params* P, T* X,
                   tp_info* info, void* ws, size_t ws_bytes, cudaStream_t st, int tc_passes, const void* Ahat) {
    return rt_solve_impl<T>(A, B, Om, l, m, n, p, P, X, info, ws, ws_bytes, st, tc_passes, false, Ahat);
}

// Adjoint of B -> X_k for the factorisation and k that the last rt_solve
// left in ws (same arguments).  Per Fourier slice, with K = A-hat V-tilde:
//   dB-hat = Q Q^H K_k S_k^{-2} V_k^H G-hat
// (U-tilde_k = B-tilde V_k S_k^{-1} = Q^H K_k S_k^{-1}).
template <typename T>
static tp_status rt_adjoint_impl(const T* G, int l, int m, int n, int p, const tp_rtsvd_params* P, T* dB, void* ws,
                                 size_t ws_bytes, cudaStream_t st, bool full) {
    TRY(rt_check<T>(l, m, n, p, P, full));
    if (!G || !dB) return TP_ERR_ARG;
    const int r_max = P->r_max, h = n / 2 + 1;
    RtWs<T> w = rt_carve<T>(ws, l, m, n, P->block, r_max, p);
    if (!ws || ((size_t)ws & 255) || ws_bytes < w.bytes) return TP_ERR_WORKSPACE;
    const long rp = (long)r_max * p;
    const int* dr = &w.st->r;
    const int* dk = &w.st->k;
    TRY(rdft<T>(G, w.Xhat, n, m, p, p, (long)m * p, nullptr, nullptr, st));
    // t = V_k^H G-hat (k x p), then t_j / sigma_j^2
    TRY(cgemm<T>(h, r_max, p, m, dk, 0, 0, 1, 0, w.Vt, r_max, (long)m * r_max, OP_C, w.Xhat, p, (long)m * p, OP_N, 0,
                 0, w.alpha, p, rp, nullptr, st));
    if (sizeof(T) == 4) TRY(alpha_corr<T>(h, w.UR, r_max, w.alpha, rp, w.st, p, st));  // as in the solve
    prof_begin(TP_KC_MISC, st);
    k_alpha<T><<<h, 256, 0, st>>>(w.sigma, r_max, w.alpha, rp, w.alpha, rp, w.st, h, l > m ? l : m, r_max, p, 2);
    TRY(launched(TP_KC_MISC, st));
    // y = K_k t (K stored transposed), z = Q^H y, dB-hat = Q z
    TRY(cgemm<T>(h, l, p, r_max, 0, 0, dk, 1, 0, w.KhT, l, (long)r_max * l, OP_T, w.alpha, p, rp, OP_N, 0, 0, w.Bhat,
                 p, (long)l * p, nullptr, st));
    TRY(cgemm<T>(h, r_max, p, l, dr, 0, 0, 1, 0, w.Q, l, (long)r_max * l, OP_R, w.Bhat, p, (long)l * p, OP_N, 0, 0,
                 w.d, p, rp, nullptr, st));
    TRY(cgemm<T>(h, l, p, r_max, 0, 0, dr, 1, 0, w.Q, l, (long)r_max * l, OP_T, w.d, p, rp, OP_N, 0, 0, w.Bhat, p,
                 (long)l * p, nullptr, st));
    return irdft<T>(w.Bhat, dB, n, l, p, p, (long)l * p, nullptr, st);
}

template <typename T>
tp_status rt_adjoint(const T* G, int l, int m, int n, int p, const tp_rtsvd_params* P, T* dB, void* ws,
                     size_t ws_bytes, cudaStream_t st) {
    return rt_adjoint_impl<T>(G, l, m, n, p, P, dB, ws, ws_bytes, st, false);
}

// ---------------------------------------------------------------------------
// T-tSVD method (Section 4.1, Eqs. (11)-(14)) through the RT-tSVD path: with
// the t-identity as the sketching tensor (Omega(:,:,1) = I, the other frontal
// slices zero, so every Fourier slice of Omega is I) and r = min(l, m), the
// block sketch spans the whole range of every A-hat slice, B-tilde = Q^H A-hat
// has the singular values of A-hat, and the discrepancy scan from k = 1
// (p = r in Eq. (kinit)) is Eq. (14)'s choice of s.  No power iterations.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_tidentity(T* Om, int m, int r) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * r; e += gridDim.x * blockDim.x) {
        const int i = e / r, j = e - i * r;
        Om[e] = i == j ? (T)1 : (T)0;  // frontal slice 1; the other slices are zeroed by a memset
    }
}

template <typename T>
static tp_rtsvd_params tt_params(int l, int m, const tp_ttsvd_params* P) {
    tp_rtsvd_params R;
    R.delta = P->delta;
    R.tau = P->tau;
    R.eps = -1.0;  // sketch to r = min(l, m) whatever the error indicator
    R.eps_rel = 0.0;
    R.r_max = l < m ? l : m;
    R.p_over = R.r_max;
    R.q_power = 0;
    R.block = 16;
    R.res_hist = P->res_hist;
    return R;
}

template <typename T>
size_t tt_ws_bytes(int l, int m, int n, int p, const tp_ttsvd_params* P) {
    if (!P) return 0;
    const tp_rtsvd_params R = tt_params<T>(l, m, P);
    if (rt_check<T>(l, m, n, p, &R, true) != TP_OK) return 0;
    const size_t rb = rt_carve<T>(nullptr, l, m, n, R.block, R.r_max, p).bytes;
    return align256(rb) + align256((size_t)n * m * R.r_max * sizeof(T));
}

template <typename T>
tp_status tt_solve(const T* A, const T* B, int l, int m, int n, int p, const tp_ttsvd_params* P, T* X,
                   tp_info* info, void* ws, size_t ws_bytes, cudaStream_t st) {
    if (!P) return TP_ERR_ARG;
    const tp_rtsvd_params R = tt_params<T>(l, m, P);
    TRY(rt_check<T>(l, m, n, p, &R, true));
    if (!A || !B || !X || !info) return TP_ERR_ARG;
    const size_t rb = align256(rt_carve<T>(nullptr, l, m, n, R.block, R.r_max, p).bytes);
    const size_t ob = (size_t)n * m * R.r_max * sizeof(T);
    if (!ws || ((size_t)ws & 255) || ws_bytes < rb + align256(ob)) return TP_ERR_WORKSPACE;
    T* Om = (T*)((char*)ws + rb);
    if (cudaMemsetAsync(Om, 0, ob, st) != cudaSuccess) return TP_ERR_CUDA;
    prof_begin(TP_KC_MISC, st);
    k_tidentity<T><<<(m * R.r_max + 255) / 256, 256, 0, st>>>(Om, m, R.r_max);
    TRY(launched(TP_KC_MISC, st));
    return rt_solve_impl<T>(A, B, Om, l, m, n, p, &R, X, info, ws, rb, st, 3, true);
}

// Adjoint of B -> X_s of the last tt_solve made with ws: the RT-tSVD adjoint
// on the factorisation the solve left in the workspace's RT-tSVD part
// (X_s = V_s S_s^{-1} U_s^T * B, Eq. (14), is linear in B at the chosen s).
template <typename T>
tp_status tt_adjoint(const T* G, int l, int m, int n, int p, const tp_ttsvd_params* P, T* dB, void* ws,
                     size_t ws_bytes, cudaStream_t st) {
    if (!P) return TP_ERR_ARG;
    const tp_rtsvd_params R = tt_params<T>(l, m, P);
    TRY(rt_check<T>(l, m, n, p, &R, true));
    const size_t rb = align256(rt_carve<T>(nullptr, l, m, n, R.block, R.r_max, p).bytes);
    if (!ws || ((size_t)ws & 255) || ws_bytes < rb) return TP_ERR_WORKSPACE;
    return rt_adjoint_impl<T>(G, l, m, n, p, &R, dB, ws, rb, st, true);
}

template tp_status tt_adjoint<float>(const float*, int, int, int, int, const tp_ttsvd_params*, float*, void*, size_t,
                                     cudaStream_t);
template tp_status tt_adjoint<double>(const double*, int, int, int, int, const tp_ttsvd_params*, double*, void*,
                                      size_t, cudaStream_t);
template size_t tt_ws_bytes<float>(int, int, int, int, const tp_ttsvd_params*);
template size_t tt_ws_bytes<double>(int, int, int, int, const tp_ttsvd_params*);
template tp_status tt_solve<float>(const float*, const float*, int, int, int, int, const tp_ttsvd_params*, float*,
                                   tp_info*, void*, size_t, cudaStream_t);
template tp_status tt_solve<double>(const double*, const double*, int, int, int, int, const tp_ttsvd_params*,
                                    double*, tp_info*, void*, size_t, cudaStream_t);
template tp_status rt_adjoint<float>(const float*, int, int, int, int, const tp_rtsvd_params*, float*, void*, size_t,
                                     cudaStream_t);
template tp_status rt_adjoint<double>(const double*, int, int, int, int, const tp_rtsvd_params*, double*, void*,
                                      size_t, cudaStream_t);
template size_t rt_ws_bytes<float>(int, int, int, int, const tp_rtsvd_params*, bool);
template size_t rt_ws_bytes<double>(int, int, int, int, const tp_rtsvd_params*, bool);
template tp_status rt_solve<float>(const float*, const float*, const float*, int, int, int, int,
                                   const tp_rtsvd_params*, float*, tp_info*, void*, size_t, cudaStream_t, int,
                                   const void*);
template tp_status rt_solve<double>(const double*, const double*, const double*, int, int, int, int,
                                    const tp_rtsvd_params*, double*, tp_info*, void*, size_t, cudaStream_t, int,
                                    const void*);

}  // namespace tp
