// Shared device helpers for the t-product library: complex arithmetic on
// float2/double2, warp and block reductions, launch bookkeeping.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "tprod.h"

namespace tp {

template <typename T> struct C2;
template <> struct C2<float> { typedef float2 type; };
template <> struct C2<double> { typedef double2 type; };
template <typename T> using cplx = typename C2<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T x, T y) {
    cplx<T> r;
    r.x = x;
    r.y = y;
    return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V> __device__ __forceinline__ V cconj(V a) { a.y = -a.y; return a; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// acc += a * b
template <typename V> __device__ __forceinline__ void cfma(V& acc, V a, V b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename V> __device__ __forceinline__ void cfmac(V& acc, V a, V b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(a.x) s) { a.x *= s; a.y *= s; return a; }
template <typename V> __device__ __forceinline__ double cabs2d(V a) {
    return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}

template <typename S> __device__ __forceinline__ S warp_sum(S v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of one value per thread over the block; every thread gets the result.
// `red` must hold blockDim.x/32 doubles.  Contains two __syncthreads().
__device__ __forceinline__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red[i];
    return t;
}

// Sum of one value per thread over the block, accumulated in the working
// precision within warps and in float64 across warps (one warp combines the
// partials); every thread gets the result.  red: 33 doubles.  Two barriers.
template <typename S>
__device__ __forceinline__ double block_sum_t(S v, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = (double)v;
    __syncthreads();
    if (w == 0) {
        double t = lane < nw ? red[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Reduce-scatter of BB (a power of two <= 32) complex values over a warp:
// returns the warp sum of entry lane / (32 / BB); the halving steps pick the
// entry index from the high lane bits.
template <typename V, int BB>
__device__ __forceinline__ V warp_reduce_scatter(V (&v)[BB]) {
    const int lane = threadIdx.x & 31;
    int cnt = BB;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (cnt > 1) {
            const bool hi = (lane & o) != 0;
            const int half = cnt >> 1;
#pragma unroll
            for (int t = 0; t < BB / 2; ++t) {
                if (t < half) {
                    V keep = hi ? v[half + t] : v[t];
                    V send = hi ? v[t] : v[half + t];
                    send.x = __shfl_xor_sync(0xffffffffu, send.x, o);
                    send.y = __shfl_xor_sync(0xffffffffu, send.y, o);
                    v[t] = cadd(keep, send);
                }
            }
            cnt = half;
        } else {
            V send = v[0];
            send.x = __shfl_xor_sync(0xffffffffu, send.x, o);
            send.y = __shfl_xor_sync(0xffffffffu, send.y, o);
            v[0] = cadd(v[0], send);
        }
    }
    return v[0];
}

template <typename V> __device__ __forceinline__ decltype(V().x) cabs2(V a) { return a.x * a.x + a.y * a.y; }

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = 1.1920928955078125e-07; };
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };

// Parseval weight of half-spectrum slice s for transform length n.
__host__ __device__ __forceinline__ double parseval_w(int s, int n) {
    return (s == 0 || 2 * s == n) ? 1.0 : 2.0;
}

// sqrt(a^2 + b^2) for Givens rotations whose arguments are norms of
// working-precision vectors: for float data the plain form cannot overflow in
// float64; double data needs the scaled hypot.
template <typename T> __device__ __forceinline__ double givens_norm(double a, double b);
template <> __device__ __forceinline__ double givens_norm<float>(double a, double b) { return sqrt(fma(a, a, b * b)); }
template <> __device__ __forceinline__ double givens_norm<double>(double a, double b) { return hypot(a, b); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// 16-byte loads of complex data: two float2 or one double2 per load.
template <typename T> struct Vec16;
template <> struct Vec16<float> { typedef float4 type; static constexpr int VW = 2; };
template <> struct Vec16<double> { typedef double2 type; static constexpr int VW = 1; };

template <typename T>
__device__ __forceinline__ void unpack(const typename Vec16<T>::type& x, cplx<T>* o);
template <> __device__ __forceinline__ void unpack<float>(const float4& x, float2* o) {
    o[0] = make_float2(x.x, x.y);
    o[1] = make_float2(x.z, x.w);
}
template <> __device__ __forceinline__ void unpack<double>(const double2& x, double2* o) { o[0] = x; }

}  // namespace tp
