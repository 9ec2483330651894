// Mode-3 DFT along the tubes of a frontal-slice-major tensor (Section 2:
// fft(A,[],3) and its inverse), real data <-> half spectrum.
//
// One CTA owns 32 tubes and all n of their entries: slice k of the 32 tubes
// is one coalesced row read, the transform runs in shared memory, and each
// output slice is one coalesced 32-element row write.  For power-of-two n two
// real tubes are packed into one complex sequence (x_a + i x_b), transformed by
// an in-place radix-2 decimation-in-time FFT and separated again; for other n
// the DFT sum is evaluated directly from a table of the n roots of unity.
// The forward kernel can also emit one float64 partial sum of squares per CTA
// (used for ||A||_F^2).
//
// A thread always handles the same tube (DFT_THREADS is a multiple of
// DFT_TILE), so its tube offset is computed once; squares are summed per
// thread in the working precision and combined in float64 across the CTA.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace tp {

constexpr int DFT_TILE = 32;
constexpr int DFT_THREADS = 256;

template <typename T> __device__ __forceinline__ void sincospi_t(T x, T* s, T* c);
template <> __device__ __forceinline__ void sincospi_t<float>(float x, float* s, float* c) { sincospif(x, s, c); }
template <> __device__ __forceinline__ void sincospi_t<double>(double x, double* s, double* c) { sincospi(x, s, c); }

__device__ __forceinline__ long tube_off(long t, int cols, long ld) {
    long r = t / cols;
    return r * ld + (t - r * cols);
}
__device__ __forceinline__ int bitrev(int x, int logn) {
    return logn ? (int)(__brev((unsigned)x) >> (32 - logn)) : 0;
}

// exp(sign * 2 pi i m / n) for m < count
template <typename T>
__device__ void fill_roots(cplx<T>* tw, int count, int n, T sign) {
    for (int m = threadIdx.x; m < count; m += blockDim.x) {
        T s, c;
        sincospi_t<T>((T)(2 * m) / (T)n, &s, &c);
        tw[m] = mk<T>(c, sign * s);
    }
}

// In-place radix-2 DIT over the 16 packed sequences z[k*16 + p] (input in
// bit-reversed order, output natural).  tw holds exp(+-2 pi i m / n), m < n/2.
template <typename T>
__device__ void fft16_inplace(cplx<T>* z, const cplx<T>* tw, int n) {
    for (int lh = 0; (1 << (lh + 1)) <= n; ++lh) {
        const int half = 1 << lh, step = n >> (lh + 1);
        for (int e = threadIdx.x; e < (n >> 1) * 16; e += blockDim.x) {
            const int p = e & 15, bf = e >> 4;
            const int j = bf & (half - 1), grp = bf >> lh;
            const int i1 = (grp << (lh + 1)) + j, i2 = i1 + half;
            cplx<T> a = z[i1 * 16 + p];
            cplx<T> b = cmul(z[i2 * 16 + p], tw[j * step]);
            z[i1 * 16 + p] = cadd(a, b);
            z[i2 * 16 + p] = csub(a, b);
        }
        __syncthreads();
    }
}

template <typename T>
__device__ void store_partial(T v, double* sumsq) {
    if (!sumsq) return;
    __shared__ double red[33];
    const double t = block_sum_t(v, red);
    if (threadIdx.x == 0) sumsq[blockIdx.x] = t;
}

static_assert(DFT_THREADS % DFT_TILE == 0, "a thread must keep one tube");

template <typename T>
__global__ void __launch_bounds__(DFT_THREADS)
k_rdft_pow2(const T* __restrict__ X, cplx<T>* __restrict__ Xh, int n, int logn, long tubes, int cols,
            long ld, long ss, double* sumsq, const int* skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<T>* z = (cplx<T>*)smraw;
    cplx<T>* tw = z + (size_t)n * 16;
    T* zf = (T*)z;
    const long t0 = (long)blockIdx.x * DFT_TILE;
    fill_roots<T>(tw, n / 2, n, (T)-1);
    const int tt = threadIdx.x & (DFT_TILE - 1), k0 = threadIdx.x / DFT_TILE, kst = blockDim.x / DFT_TILE;
    const bool live = t0 + tt < tubes;
    const T* xt = X + (live ? tube_off(t0 + tt, cols, ld) : 0);
    T acc = 0;
    // LB loads in flight per thread before any is used (the tube entries are
    // one strided row each: the kernel is bound by how many rows are in flight)
    constexpr int LB = sizeof(T) == 4 ? 32 : 16;
    for (int kb = k0; kb < n; kb += LB * kst) {
        T v[LB];
#pragma unroll
        for (int j = 0; j < LB; ++j) {
            const int k = kb + j * kst;
            v[j] = (live && k < n) ? __ldcs(xt + (long)k * ss) : (T)0;
        }
#pragma unroll
        for (int j = 0; j < LB; ++j) {
            const int k = kb + j * kst;
            if (k < n) {
                acc = fma(v[j], v[j], acc);
                zf[((size_t)bitrev(k, logn) * 16 + (tt & 15)) * 2 + (tt >> 4)] = v[j];
            }
        }
    }
    __syncthreads();
    fft16_inplace<T>(z, tw, n);
    const int h = n / 2 + 1;
    for (int e = threadIdx.x; e < h * DFT_TILE; e += blockDim.x) {
        const int s = e >> 5, tt = e & 31;
        const long t = t0 + tt;
        if (t >= tubes) continue;
        const int p = tt & 15;
        cplx<T> zs = z[s * 16 + p];
        cplx<T> zc = cconj(z[((n - s) & (n - 1)) * 16 + p]);
        cplx<T> o;
        if (tt < 16) o = mk<T>((zs.x + zc.x) * (T)0.5, (zs.y + zc.y) * (T)0.5);
        else o = mk<T>((zs.y - zc.y) * (T)0.5, -(zs.x - zc.x) * (T)0.5);
        Xh[(long)s * tubes + t] = o;
    }
    store_partial<T>(acc, sumsq);
}

// ---- register DFTs of 4, 16 and 32 points (the n = 16 Q kernels below) --------
template <typename T>
__device__ __forceinline__ void dft4f(cplx<T>& x0, cplx<T>& x1, cplx<T>& x2, cplx<T>& x3) {
    // forward 4-point DFT in place: X_k = sum_n x_n exp(-2 pi i n k / 4)
    const cplx<T> t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = csub(x1, x3);
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = mk<T>(t1.x + t3.y, t1.y - t3.x);  // t1 - i t3
    x3 = mk<T>(t1.x - t3.y, t1.y + t3.x);  // t1 + i t3
}

// forward 16-point DFT of v in place, natural order in and out (4 x 4 split)
template <typename T>
__device__ __forceinline__ void dft16f(cplx<T> (&v)[16]) {
    const T c8 = (T)0.92387953251128675613, s8 = (T)0.38268343236508977173, h2 = (T)0.70710678118654752440;
    // step 1: for each n2, the 4-point DFT over n1 of v[4 n1 + n2] -> a[k1][n2] kept at v[4 k1 + n2]
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4f<T>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    // step 2: twiddles exp(-2 pi i n2 k1 / 16), n2 k1 in {1, 2, 3, 2, 4, 6, 3, 6, 9}
    auto tw = [](cplx<T> a, T c, T s) { return mk<T>(a.x * c - a.y * s, a.x * s + a.y * c); };  // a (c + i s)
    v[4 * 1 + 1] = tw(v[5], c8, -s8);
    v[4 * 1 + 2] = tw(v[6], h2, -h2);
    v[4 * 1 + 3] = tw(v[7], s8, -c8);
    v[4 * 2 + 1] = tw(v[9], h2, -h2);
    v[4 * 2 + 2] = mk<T>(v[10].y, -v[10].x);  // times -i
    v[4 * 2 + 3] = tw(v[11], -h2, -h2);
    v[4 * 3 + 1] = tw(v[13], s8, -c8);
    v[4 * 3 + 2] = tw(v[14], -h2, -h2);
    v[4 * 3 + 3] = tw(v[15], -c8, s8);
    // step 3: for each k1, the 4-point DFT over n2 -> X[k1 + 4 k2]
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4f<T>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // v[4 k1 + k2] holds X[k1 + 4 k2]: transpose the 4 x 4 index
    cplx<T> o[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) o[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = o[i];
}

// forward 32-point DFT of v in place, natural order in and out: the 16-point
// DFTs of the even and odd entries, combined with exp(-2 pi i k / 32)
template <typename T>
__device__ __forceinline__ void dft32f(cplx<T> (&v)[32]) {
    // cos and sin of 2 pi k / 32, k = 0 .. 7
    const T c1 = (T)0.98078528040323044913, s1 = (T)0.19509032201612826785;
    const T c2 = (T)0.92387953251128675613, s2 = (T)0.38268343236508977173;
    const T c3 = (T)0.83146961230254523708, s3 = (T)0.55557023301960222474, h2 = (T)0.70710678118654752440;
    const T C[8] = {(T)1, c1, c2, c3, h2, s3, s2, s1}, S[8] = {(T)0, s1, s2, s3, h2, c3, c2, c1};
    cplx<T> e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        e[i] = v[2 * i];
        o[i] = v[2 * i + 1];
    }
    dft16f<T>(e);
    dft16f<T>(o);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        // exp(-2 pi i k / 32) = c - i s; k >= 8 turns by a further -pi / 2
        const T c = k < 8 ? C[k] : -S[k - 8], sn = k < 8 ? S[k] : C[k - 8];
        const cplx<T> t = mk<T>(o[k].x * c + o[k].y * sn, o[k].y * c - o[k].x * sn);
        v[k] = cadd(e[k], t);
        v[k + 16] = csub(e[k], t);
    }
}
template <typename T, int Q> struct DftQ;
template <typename T> struct DftQ<T, 16> {
    static __device__ __forceinline__ void run(cplx<T> (&v)[16]) { dft16f<T>(v); }
};
template <typename T> struct DftQ<T, 32> {
    static __device__ __forceinline__ void run(cplx<T> (&v)[32]) { dft32f<T>(v); }
};

// ---- n = 16 Q (Q = 16: n = 256; Q = 32: n = 512) ------------------------------
// x_t with t = Q t1 + t2 (t1 < 16, t2 < Q), X_k with k = k1 + 16 k2:
//   X[k1 + 16 k2] = sum_t2 exp(-2 pi i t2 k2 / Q) exp(-2 pi i t2 k1 / n)
//                   sum_t1 exp(-2 pi i t1 k1 / 16) x[Q t1 + t2].
// Thread (seq, j) of the 16 per packed sequence does the 16-point DFTs over t1
// for t2 = j, j + 16, ... (Q / 16 of them), applies the twiddles, and then the
// Q-point DFT over t2 for k1 = j, all in registers.  The three shared-memory
// phases (real input [t][tube], twiddled partial DFTs [seq][k1][t2], packed
// spectrum [k][seq]) share one buffer, each read into registers behind a
// barrier before the next is written, so that several CTAs fit on an SM.
template <int Q> struct Rdft16Q {
    static constexpr int n = 16 * Q, TS = Q + 1, ZS = 17;
    template <typename T> static constexpr size_t region() {
        const size_t b = (size_t)256 * TS * 2 * sizeof(T), c = (size_t)n * ZS * 2 * sizeof(T);
        return b > c ? b : c;
    }
    template <typename T> static constexpr size_t smem() { return (size_t)n * 2 * sizeof(T) + region<T>(); }
};

template <typename T, int Q>
__global__ void __launch_bounds__(DFT_THREADS, sizeof(T) == 4 ? (Q == 16 ? 5 : 3) : 1)
k_rdft_16q(const T* __restrict__ X, cplx<T>* __restrict__ Xh, long tubes, int cols, long ld, long ss, double* sumsq,
           const int* skip) {
    if (skip && *skip) return;
    typedef Rdft16Q<Q> R;
    constexpr int n = R::n, TS = R::TS, ZS = R::ZS, h = n / 2 + 1;
    constexpr int NT = DFT_THREADS;  // compile-time strides: the index arithmetic folds into constants
    static_assert(NT == 256, "16 packed sequences x 16 threads");
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<T>* tw = (cplx<T>*)smraw;                 // n roots exp(-2 pi i m / n)
    cplx<T>* zp = tw + n;                          // phase 1: packed input [t][seq], row stride 17
    cplx<T>* zt = zp;                              // phase 2: [seq][k1][t2], row stride Q + 1
    cplx<T>* z = zp;                               // phase 3: packed spectrum [k][seq], row stride 17
    const int tid = threadIdx.x;
    const long t0 = (long)blockIdx.x * DFT_TILE;
    {
        const T step = (T)2 / (T)n;  // exact for a power of two: the argument 2 m / n without a division
        for (int m = tid; m < n; m += NT) {
            T sn, cs;
            sincospi_t<T>((T)m * step, &sn, &cs);
            tw[m] = mk<T>(cs, -sn);
        }
    }
    // phase 1: thread (row group kr, pair p) loads tubes p and p + 16 (the real and imaginary parts of packed
    // sequence p) at rows kr, kr + 16, ...; a half-warp reads 16 consecutive tubes of one row
    const int p = tid & 15, kr = tid >> 4;
    T acc = 0;
    {
        const bool la = t0 + p < tubes, lb = t0 + p + 16 < tubes;
        const T* xa = X + (la ? tube_off(t0 + p, cols, ld) : 0);
        const T* xb = X + (lb ? tube_off(t0 + p + 16, cols, ld) : 0);
        constexpr int RPT = n / 16;                  // rows per thread
        constexpr int LB = RPT > 16 ? 16 : RPT;      // row pairs in flight per thread
#pragma unroll 1
        for (int rb = 0; rb < RPT; rb += LB) {
            T va[LB], vb[LB];
#pragma unroll
            for (int i = 0; i < LB; ++i) {
                const long off = (long)(kr + 16 * (rb + i)) * ss;
                va[i] = la ? __ldcs(xa + off) : (T)0;
                vb[i] = lb ? __ldcs(xb + off) : (T)0;
            }
#pragma unroll
            for (int i = 0; i < LB; ++i) {
                acc = fma(va[i], va[i], acc);
                acc = fma(vb[i], vb[i], acc);
                zp[(kr + 16 * (rb + i)) * ZS + p] = mk<T>(va[i], vb[i]);
            }
        }
    }
    __syncthreads();
    const int seq = tid >> 4, j = tid & 15;
    {
        // 16-point DFTs over t1 of x[Q t1 + t2], t2 = j + 16 u
        cplx<T> v[Q / 16][16];
#pragma unroll
        for (int u = 0; u < Q / 16; ++u)
#pragma unroll
            for (int t1 = 0; t1 < 16; ++t1) v[u][t1] = zp[(Q * t1 + j + 16 * u) * ZS + seq];
        __syncthreads();  // the input is read: the buffer takes the partial DFTs
#pragma unroll
        for (int u = 0; u < Q / 16; ++u) {
            const int t2 = j + 16 * u;
            dft16f<T>(v[u]);
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) zt[(seq * 16 + k1) * TS + t2] = cmul(v[u][k1], tw[(t2 * k1) & (n - 1)]);
        }
    }
    __syncthreads();
    {
        // Q-point DFT over t2 for k1 = j: X[j + 16 k2]
        cplx<T> v[Q];
#pragma unroll
        for (int t2 = 0; t2 < Q; ++t2) v[t2] = zt[(seq * 16 + j) * TS + t2];
        __syncthreads();  // the partial DFTs are read: the buffer takes the spectrum
        DftQ<T, Q>::run(v);
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) z[(j + 16 * k2) * ZS + seq] = v[k2];
    }
    __syncthreads();
    {
        // separate the two real tubes of each packed sequence: thread (row group, tube tq) writes
        // slices s = tid / 32 + 8 i of tube tq; tq < 16 takes (Z_s + conj Z_{n-s}) / 2, the others
        // (Z_s - conj Z_{n-s}) / 2i, branch-free
        const int tq = tid & 31, q = tq & 15, s0 = tid >> 5;
        const long t = t0 + tq;
        const T sg = tq < 16 ? (T)1 : (T)-1;
        if (t < tubes) {
            cplx<T>* dst = Xh + t + (long)s0 * tubes;
            const long dstep = 8 * tubes;
#pragma unroll 4
            for (int s = s0; s < h; s += NT / 32, dst += dstep) {
                const cplx<T> zs = z[s * ZS + q];
                const cplx<T> zc = z[((n - s) & (n - 1)) * ZS + q];
                const T ux = fma(sg, zc.x, zs.x), uy = fma(-sg, zc.y, zs.y);  // Z_s +- conj Z_{n-s}
                *dst = tq < 16 ? mk<T>(ux * (T)0.5, uy * (T)0.5) : mk<T>(uy * (T)0.5, -ux * (T)0.5);
            }
        }
    }
    store_partial<T>(acc, sumsq);
}

// Inverse for n = 256: the half spectra of 32 tubes become 16 packed full
// spectra Z = X_a + i X_b, transformed back by the 16 x 16 split with
// conjugated roots (the inverse DFT is conj(DFT(conj(Z)))), scaled by 1/n.
template <typename T>
__global__ void __launch_bounds__(DFT_THREADS)
k_irdft_256(const cplx<T>* __restrict__ Xh, T* __restrict__ X, long tubes, int cols, long ld, long ss,
            const int* skip) {
    if (skip && *skip) return;
    constexpr int n = 256, TS = 17;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<T>* tw = (cplx<T>*)smraw;          // 256 roots exp(-2 pi i m / 256)
    cplx<T>* zt = tw + n;                   // [seq][k1][n2], row stride 17
    cplx<T>* z = zt + 16 * 16 * TS;         // conj of the packed spectrum, then the packed signal: [k][seq]
    const long t0 = (long)blockIdx.x * DFT_TILE;
    fill_roots<T>(tw, n, n, (T)-1);
    const int h = n / 2 + 1;
    constexpr int LB = sizeof(T) == 4 ? 8 : 4;
    for (int e0 = threadIdx.x; e0 < h * 16; e0 += LB * blockDim.x) {
        cplx<T> xa[LB], xb[LB];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int e = e0 + u * blockDim.x;
            const int s = e >> 4, p = e & 15;
            const long ta = t0 + p, tb = t0 + p + 16;
            xa[u] = (e < h * 16 && ta < tubes) ? Xh[(long)s * tubes + ta] : mk<T>(0, 0);
            xb[u] = (e < h * 16 && tb < tubes) ? Xh[(long)s * tubes + tb] : mk<T>(0, 0);
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e >= h * 16) break;
            const int s = e >> 4, p = e & 15;
            cplx<T> a = xa[u], b = xb[u];
            const bool self = (s == 0) || (2 * s == n);
            if (self) { a.y = 0; b.y = 0; }
            // conj(Z[s]) and conj(Z[n - s]), Z = X_a + i X_b with X(n - s) = conj(X(s))
            z[s * TS + p] = mk<T>(a.x - b.y, -(a.y + b.x));
            if (!self) z[(n - s) * TS + p] = mk<T>(a.x + b.y, -(b.x - a.y));
        }
    }
    __syncthreads();
    const int seq = threadIdx.x >> 4, j = threadIdx.x & 15;
    {
        cplx<T> v[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) v[n1] = z[(16 * n1 + j) * TS + seq];
        dft16f<T>(v);
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) zt[(seq * 16 + k1) * TS + j] = cmul(v[k1], tw[(j * k1) & (n - 1)]);
    }
    __syncthreads();
    {
        cplx<T> v[16];
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) v[n2] = zt[(seq * 16 + j) * TS + n2];
        dft16f<T>(v);
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) z[(j + 16 * k2) * TS + seq] = v[k2];  // conj of the packed signal
    }
    __syncthreads();
    const T inv = (T)1 / (T)n;
    const int tt = threadIdx.x & (DFT_TILE - 1), k0 = threadIdx.x / DFT_TILE, kst = blockDim.x / DFT_TILE;
    if (t0 + tt < tubes) {
        T* xt = X + tube_off(t0 + tt, cols, ld);
#pragma unroll 8
        for (int k = k0; k < n; k += kst) {
            const cplx<T> v = z[k * TS + (tt & 15)];
            xt[(long)k * ss] = (tt < 16 ? v.x : -v.y) * inv;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(DFT_THREADS)
k_rdft_direct(const T* __restrict__ X, cplx<T>* __restrict__ Xh, int n, long tubes, int cols,
              long ld, long ss, double* sumsq, const int* skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<T>* tw = (cplx<T>*)smraw;
    T* x = (T*)(tw + n);
    const long t0 = (long)blockIdx.x * DFT_TILE;
    fill_roots<T>(tw, n, n, (T)-1);
    const int tt = threadIdx.x & (DFT_TILE - 1), k0 = threadIdx.x / DFT_TILE, kst = blockDim.x / DFT_TILE;
    const bool live = t0 + tt < tubes;
    const T* xt = X + (live ? tube_off(t0 + tt, cols, ld) : 0);
    T acc = 0;
#pragma unroll 4
    for (int k = k0; k < n; k += kst) {
        const T v = live ? xt[(long)k * ss] : (T)0;
        acc = fma(v, v, acc);
        x[k * DFT_TILE + tt] = v;
    }
    __syncthreads();
    const int h = n / 2 + 1;
    for (int e = threadIdx.x; e < h * DFT_TILE; e += blockDim.x) {
        const int s = e >> 5, tt = e & 31;
        const long t = t0 + tt;
        cplx<T> o = mk<T>(0, 0);
        int idx = 0;
        for (int k = 0; k < n; ++k) {
            const T v = x[k * DFT_TILE + tt];
            o.x = fma(v, tw[idx].x, o.x);
            o.y = fma(v, tw[idx].y, o.y);
            idx += s;
            if (idx >= n) idx -= n;
        }
        if (t < tubes) Xh[(long)s * tubes + t] = o;
    }
    store_partial<T>(acc, sumsq);
}

template <typename T>
__global__ void __launch_bounds__(DFT_THREADS)
k_irdft_pow2(const cplx<T>* __restrict__ Xh, T* __restrict__ X, int n, int logn, long tubes, int cols,
             long ld, long ss, const int* skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<T>* z = (cplx<T>*)smraw;
    cplx<T>* tw = z + (size_t)n * 16;
    const long t0 = (long)blockIdx.x * DFT_TILE;
    fill_roots<T>(tw, n / 2, n, (T)1);
    const int h = n / 2 + 1;
    // LB pairs of spectrum loads in flight per thread before any is used
    constexpr int LB = sizeof(T) == 4 ? 8 : 4;
    for (int e0 = threadIdx.x; e0 < h * 16; e0 += LB * blockDim.x) {
        cplx<T> xa[LB], xb[LB];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int e = e0 + u * blockDim.x;
            const int s = e >> 4, p = e & 15;
            const long ta = t0 + p, tb = t0 + p + 16;
            xa[u] = (e < h * 16 && ta < tubes) ? Xh[(long)s * tubes + ta] : mk<T>(0, 0);
            xb[u] = (e < h * 16 && tb < tubes) ? Xh[(long)s * tubes + tb] : mk<T>(0, 0);
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e >= h * 16) break;
            const int s = e >> 4, p = e & 15;
            cplx<T> a = xa[u], b = xb[u];
            const bool self = (s == 0) || (2 * s == n);
            if (self) { a.y = 0; b.y = 0; }
            z[bitrev(s, logn) * 16 + p] = mk<T>(a.x - b.y, a.y + b.x);
            if (!self) z[bitrev(n - s, logn) * 16 + p] = mk<T>(a.x + b.y, b.x - a.y);
        }
    }
    __syncthreads();
    fft16_inplace<T>(z, tw, n);
    const T inv = (T)1 / (T)n;
    const int tt = threadIdx.x & (DFT_TILE - 1), k0 = threadIdx.x / DFT_TILE, kst = blockDim.x / DFT_TILE;
    if (t0 + tt < tubes) {
        T* xt = X + tube_off(t0 + tt, cols, ld);
#pragma unroll 8
        for (int k = k0; k < n; k += kst) {
            const cplx<T> v = z[k * 16 + (tt & 15)];
            xt[(long)k * ss] = (tt < 16 ? v.x : v.y) * inv;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(DFT_THREADS)
k_irdft_direct(const cplx<T>* __restrict__ Xh, T* __restrict__ X, int n, long tubes, int cols,
               long ld, long ss, const int* skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<T>* tw = (cplx<T>*)smraw;
    cplx<T>* xs = tw + n;
    const long t0 = (long)blockIdx.x * DFT_TILE;
    fill_roots<T>(tw, n, n, (T)1);
    const int h = n / 2 + 1;
    for (int e = threadIdx.x; e < h * DFT_TILE; e += blockDim.x) {
        const int s = e >> 5, tt = e & 31;
        const long t = t0 + tt;
        cplx<T> v = mk<T>(0, 0);
        if (t < tubes) v = Xh[(long)s * tubes + t];
        if (s == 0 || 2 * s == n) v.y = 0;
        xs[e] = v;
    }
    __syncthreads();
    const T inv = (T)1 / (T)n;
    const int tt = threadIdx.x & (DFT_TILE - 1), k0 = threadIdx.x / DFT_TILE, kst = blockDim.x / DFT_TILE;
    const bool live = t0 + tt < tubes;
    T* xt = X + (live ? tube_off(t0 + tt, cols, ld) : 0);
    for (int k = k0; k < n; k += kst) {
        T acc = xs[tt].x;  // slice 0
        int idx = k;
        for (int s = 1; s < h; ++s) {
            const cplx<T> v = xs[s * DFT_TILE + tt];
            const T wgt = (2 * s == n) ? (T)1 : (T)2;
            acc += wgt * (v.x * tw[idx].x - v.y * tw[idx].y);
            idx += k;
            if (idx >= n) idx -= n;
        }
        if (live) xt[(long)k * ss] = acc * inv;
    }
}

static inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
static inline int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

int rdft_parts(int rows, int cols) { return (int)(((long)rows * cols + DFT_TILE - 1) / DFT_TILE); }

size_t rdft_smem(int n, size_t elem) {
    const size_t c = 2 * elem;
    if (is_pow2(n)) return ((size_t)n * 16 + n / 2) * c;
    const size_t fwd = (size_t)n * c + (size_t)n * DFT_TILE * elem;
    const size_t inv = (size_t)n * c + (size_t)(n / 2 + 1) * DFT_TILE * c;
    return fwd > inv ? fwd : inv;
}

template <typename K>
static tp_status prep(K kern, size_t smem) {
    if (smem_optin((const void*)kern, smem) != TP_OK) return TP_ERR_CUDA;
    return TP_OK;
}

template <typename T>
tp_status rdft(const T* X, void* Xh, int n, int rows, int cols, long ld, long ss, double* sumsq,
               const int* skip, cudaStream_t st) {
    const long tubes = (long)rows * cols;
    if (tubes == 0) return TP_OK;
    const unsigned grid = (unsigned)((tubes + DFT_TILE - 1) / DFT_TILE);
    const size_t smem = rdft_smem(n, sizeof(T));
    if (n == 256 || n == 512) {
        const size_t sm = n == 256 ? Rdft16Q<16>::smem<T>() : Rdft16Q<32>::smem<T>();
        auto kern = n == 256 ? k_rdft_16q<T, 16> : k_rdft_16q<T, 32>;
        if (prep(kern, sm) != TP_OK) return TP_ERR_CUDA;
        prof_begin(TP_KC_DFT, st);
        kern<<<grid, DFT_THREADS, sm, st>>>(X, (cplx<T>*)Xh, tubes, cols, ld, ss, sumsq, skip);
    } else if (is_pow2(n)) {
        if (prep(k_rdft_pow2<T>, smem) != TP_OK) return TP_ERR_CUDA;
        prof_begin(TP_KC_DFT, st);
        k_rdft_pow2<T><<<grid, DFT_THREADS, smem, st>>>(X, (cplx<T>*)Xh, n, ilog2(n), tubes, cols, ld, ss,
                                                         sumsq, skip);
    } else {
        if (prep(k_rdft_direct<T>, smem) != TP_OK) return TP_ERR_CUDA;
        prof_begin(TP_KC_DFT, st);
        k_rdft_direct<T><<<grid, DFT_THREADS, smem, st>>>(X, (cplx<T>*)Xh, n, tubes, cols, ld, ss, sumsq, skip);
    }
    return launched(TP_KC_DFT, st);
}

template <typename T>
tp_status irdft(const void* Xh, T* X, int n, int rows, int cols, long ld, long ss, const int* skip,
                cudaStream_t st) {
    const long tubes = (long)rows * cols;
    if (tubes == 0) return TP_OK;
    const unsigned grid = (unsigned)((tubes + DFT_TILE - 1) / DFT_TILE);
    const size_t smem = rdft_smem(n, sizeof(T));
    if (n == 256) {
        const size_t sm256 = (size_t)(256 + 2 * 16 * 16 * 17) * 2 * sizeof(T);
        if (prep(k_irdft_256<T>, sm256) != TP_OK) return TP_ERR_CUDA;
        prof_begin(TP_KC_DFT, st);
        k_irdft_256<T><<<grid, DFT_THREADS, sm256, st>>>((const cplx<T>*)Xh, X, tubes, cols, ld, ss, skip);
    } else if (is_pow2(n)) {
        if (prep(k_irdft_pow2<T>, smem) != TP_OK) return TP_ERR_CUDA;
        prof_begin(TP_KC_DFT, st);
        k_irdft_pow2<T><<<grid, DFT_THREADS, smem, st>>>((const cplx<T>*)Xh, X, n, ilog2(n), tubes, cols, ld,
                                                          ss, skip);
    } else {
        if (prep(k_irdft_direct<T>, smem) != TP_OK) return TP_ERR_CUDA;
        prof_begin(TP_KC_DFT, st);
        k_irdft_direct<T><<<grid, DFT_THREADS, smem, st>>>((const cplx<T>*)Xh, X, n, tubes, cols, ld, ss, skip);
    }
    return launched(TP_KC_DFT, st);
}

// ||X||_F^2 from a half spectrum (h = n/2 + 1 slices of rows x cols), in the
// same rdft_parts(rows, cols) partial sums the forward transform writes:
// Parseval, (1/n) sum_s w_s ||X-hat_s||^2.  Partial b covers the entries
// DFT_TILE b .. DFT_TILE (b+1) - 1 of every slice; the 256 threads of its CTA
// take the 32 entries of eight slices at a time (their loads independent), and
// the sum runs in a fixed order (per thread in the working precision, across
// threads in float64).
template <typename T>
__global__ void __launch_bounds__(256) k_norm2_hat(const cplx<T>* __restrict__ Xh, int n, int h, long rc, int nparts,
                                                   double* parts) {
    __shared__ double red[33];
    const int b = blockIdx.x, t = threadIdx.x & (DFT_TILE - 1), g = threadIdx.x / DFT_TILE;
    const int ng = blockDim.x / DFT_TILE;
    const long e = (long)b * DFT_TILE + t;
    double acc = 0.0;
    if (e < rc)
#pragma unroll 4
        for (int s = g; s < h; s += ng) acc += parseval_w(s, n) * (double)cabs2(__ldg(Xh + (long)s * rc + e));
    acc = block_sum_t(acc, red);
    if (threadIdx.x == 0) parts[b] = acc / (double)n;
}

template <typename T>
tp_status norm2_hat(const void* Xh, int n, int rows, int cols, double* parts, cudaStream_t st) {
    const int np = rdft_parts(rows, cols), h = n / 2 + 1;
    prof_begin(TP_KC_DFT, st);
    k_norm2_hat<T><<<np, 256, 0, st>>>((const cplx<T>*)Xh, n, h, (long)rows * cols, np, parts);
    return launched(TP_KC_DFT, st);
}
template tp_status norm2_hat<float>(const void*, int, int, int, double*, cudaStream_t);
template tp_status norm2_hat<double>(const void*, int, int, int, double*, cudaStream_t);

template tp_status rdft<float>(const float*, void*, int, int, int, long, long, double*, const int*, cudaStream_t);
template tp_status rdft<double>(const double*, void*, int, int, int, long, long, double*, const int*, cudaStream_t);
template tp_status irdft<float>(const void*, float*, int, int, int, long, long, const int*, cudaStream_t);
template tp_status irdft<double>(const void*, double*, int, int, int, long, long, const int*, cudaStream_t);

}  // namespace tp
