// Gradients with respect to the tube weights c of a separable operator
// A(:,:,k) = c_k T.  Every Fourier slice of A is c-hat_s T, and the subspaces
// the solvers build from a slice (the RT-tSVD sketch and its power
// iterations, the tGKB Krylov space, the singular vectors) are those of T,
// so with the discrete choices of a solve held fixed its solution is
// X-hat_s = M_s B-hat_s / c-hat_s (M_s free of c) for the truncated methods,
// and z(lam / |c-hat_s|^2) / c-hat_s for the projected Tikhonov solution with
// damping lam (z the solution for T).  With gamma_s = <G-hat_s, X-hat_s> and
// the Tikhonov term t_s = 2 lam Re<G-hat_s, dX-hat_s/dlam> (zero otherwise),
// Parseval and dc-hat_s = sum_k dc_k w^{sk} (w = exp(-2 pi i / n)) give
//   dL/dc_k = -(1/n) sum_{s<n} Re( (gamma_s + t_s) / c-hat_s * w^{sk} ),
// summed here over the half spectrum with the Parseval weights (slices s and
// n - s contribute complex conjugates).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace tp {

// gamma[s] = sum_e conj(Gh[s, e]) Xh[s, e] over the `per` entries of slice s:
// products in the working precision, float64 sums in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_sep_gamma(const cplx<T>* Xh, const cplx<T>* Gh, long per, double2* gamma) {
    __shared__ double red[32];
    const int s = blockIdx.x;
    const cplx<T>* x = Xh + (long)s * per;
    const cplx<T>* g = Gh + (long)s * per;
    double re = 0.0, im = 0.0;
    for (long e = threadIdx.x; e < per; e += blockDim.x) {
        const cplx<T> a = g[e], b = x[e];
        re += (double)(a.x * b.x + a.y * b.y);
        im += (double)(a.x * b.y - a.y * b.x);
    }
    re = block_sum(re, red);
    im = block_sum(im, red);
    if (threadIdx.x == 0) gamma[s] = make_double2(re, im);
}

// One CTA: the twiddles w^j (j < n), c-hat_s for the h half-spectrum slices,
// a_s = -(w_s / n) (gamma_s + add_s) / c-hat_s, then dc_k = sum_s Re(a_s w^{sk}).
// A slice with c-hat_s = 0 contributes nothing (its forward solve divides by
// zero).  Shared memory: (n + h) double2.
__global__ void __launch_bounds__(256) k_grad_c(const double* c, int n, const double2* gamma, const double* add,
                                                double* dc) {
    extern __shared__ double2 gsm[];
    double2* tw = gsm;
    double2* a = gsm + n;
    const int h = n / 2 + 1;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)j / (double)n, &sn, &cs);
        tw[j] = make_double2(cs, -sn);
    }
    __syncthreads();
    for (int s = threadIdx.x; s < h; s += blockDim.x) {
        double cr = 0.0, ci = 0.0;
        int idx = 0;  // s k mod n
        for (int k = 0; k < n; ++k) {
            const double2 w = tw[idx];
            cr = fma(c[k], w.x, cr);
            ci = fma(c[k], w.y, ci);
            idx += s;
            if (idx >= n) idx -= n;
        }
        const double gr = gamma[s].x + (add ? add[s] : 0.0), gi = gamma[s].y;
        const double den = cr * cr + ci * ci;
        const double f = den > 0.0 ? -parseval_w(s, n) / ((double)n * den) : 0.0;
        a[s] = make_double2(f * (gr * cr + gi * ci), f * (gi * cr - gr * ci));
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double acc = 0.0;
        int idx = 0;  // s k mod n
        for (int s = 0; s < h; ++s) {
            const double2 w = tw[idx];
            acc = fma(a[s].x, w.x, acc);
            acc = fma(-a[s].y, w.y, acc);
            idx += k;
            if (idx >= n) idx -= n;
        }
        dc[k] = acc;
    }
}

template <typename T>
tp_status sep_gamma(const void* Xh, const void* Gh, int h, long per, double2* gamma, cudaStream_t st) {
    prof_begin(TP_KC_MISC, st);
    k_sep_gamma<T><<<h, 256, 0, st>>>((const cplx<T>*)Xh, (const cplx<T>*)Gh, per, gamma);
    return launched(TP_KC_MISC, st);
}

tp_status grad_c(const double* c, int n, const double2* gamma, const double* add, double* dc, cudaStream_t st) {
    const size_t smem = (size_t)(n + n / 2 + 1) * sizeof(double2);
    prof_begin(TP_KC_MISC, st);
    k_grad_c<<<1, 256, smem, st>>>(c, n, gamma, add, dc);
    return launched(TP_KC_MISC, st);
}

// A(:,:,k) = c_k T, the product formed in float64 and rounded once.
template <typename T>
__global__ void k_sep_operator(const T* Tm, const double* c, long lm, int n, T* A) {
    const long total = (long)n * lm;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long k = e / lm, ij = e - k * lm;
        A[e] = (T)(c[k] * (double)Tm[ij]);
    }
}

template <typename T>
tp_status sep_operator(const T* Tm, const double* c, int l, int m, int n, T* A, cudaStream_t st) {
    if (!Tm || !c || !A || l < 1 || m < 1 || n < 1) return TP_ERR_ARG;
    const long total = (long)n * l * m;
    const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
    prof_begin(TP_KC_MISC, st);
    k_sep_operator<T><<<blocks, 256, 0, st>>>(Tm, c, (long)l * m, n, A);
    return launched(TP_KC_MISC, st);
}

template tp_status sep_operator<float>(const float*, const double*, int, int, int, float*, cudaStream_t);
template tp_status sep_operator<double>(const double*, const double*, int, int, int, double*, cudaStream_t);

template tp_status sep_gamma<float>(const void*, const void*, int, long, double2*, cudaStream_t);
template tp_status sep_gamma<double>(const void*, const void*, int, long, double2*, cudaStream_t);

static bool grad_dims_ok(int m, int n, int p) {
    return m >= 1 && n >= 1 && p >= 1 && m <= 4096 && p <= 4096 && n <= GRAD_MAX_N;
}

template <typename T>
size_t sep_ws_bytes(int m, int n, int p) {
    if (!grad_dims_ok(m, n, p)) return 0;
    const size_t h = n / 2 + 1, per = (size_t)m * p;
    Carver cv(nullptr, 0);
    cv.take<cplx<T>>(h * per);
    cv.take<cplx<T>>(h * per);
    cv.take<double2>(h);
    return cv.off;
}

template <typename T>
tp_status sep_grad(const T* X, const T* G, const double* c, int m, int n, int p, double* dc, void* ws,
                   size_t ws_bytes, cudaStream_t st) {
    if (!grad_dims_ok(m, n, p) || !X || !G || !c || !dc) return TP_ERR_ARG;
    const int h = n / 2 + 1;
    const long per = (long)m * p;
    Carver cv(ws, ws_bytes);
    cplx<T>* Xh = cv.take<cplx<T>>((size_t)h * per);
    cplx<T>* Gh = cv.take<cplx<T>>((size_t)h * per);
    double2* gamma = cv.take<double2>(h);
    if (!ws || ((size_t)ws & 255) || ws_bytes < cv.off) return TP_ERR_WORKSPACE;
    tp_status e = rdft<T>(X, Xh, n, m, p, p, per, nullptr, nullptr, st);
    if (e != TP_OK) return e;
    e = rdft<T>(G, Gh, n, m, p, p, per, nullptr, nullptr, st);
    if (e != TP_OK) return e;
    e = sep_gamma<T>(Xh, Gh, h, per, gamma, st);
    if (e != TP_OK) return e;
    return grad_c(c, n, gamma, nullptr, dc, st);
}

template size_t sep_ws_bytes<float>(int, int, int);
template size_t sep_ws_bytes<double>(int, int, int);
template tp_status sep_grad<float>(const float*, const float*, const double*, int, int, int, double*, void*, size_t,
                                   cudaStream_t);
template tp_status sep_grad<double>(const double*, const double*, const double*, int, int, int, double*, void*,
                                    size_t, cudaStream_t);

}  // namespace tp
