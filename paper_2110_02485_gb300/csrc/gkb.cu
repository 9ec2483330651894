// tGKB (Algorithm 4) and the tGKB / Tikhonov-tGKB methods on the half spectrum.
//
// Every t-operation of Algorithm 4 is facewise in the Fourier domain, so each
// Fourier slice runs its own Golub-Kahan bidiagonalisation; the slices are
// coupled only by the discrepancy test, whose residual is the Parseval sum of
// the per-slice least-squares residuals.  The whole iteration is one
// persistent cooperative launch with one CTA per slice: after each step a CTA
// publishes its residual and waits (bounded) until all slices have done the
// step, then every CTA evaluates the same fixed-order sum and so takes the
// same stop decision.  Normalize's coefficients are non-negative reals per
// slice, so the projected problem of each slice is a real lower-bidiagonal
// least-squares problem, solved incrementally by Givens rotations (float64).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace tp {

constexpr int GKB_KMAX = 512;
constexpr int GKB_MAX_RHS = 1024;  // lateral slices of B per tgkb_solve call

struct GkbShared {
    double res[GKB_KMAX + 1];   // global residual after step i
    double rho[GKB_KMAX], theta[GKB_KMAX + 1], phi[GKB_KMAX];
    double y[GKB_KMAX];
};

template <typename T>
__device__ void mv_h(const cplx<T>* __restrict__ A, int l, int m, const cplx<T>* q, cplx<T>* u) {
    // u[j] = sum_i conj(A[i][j]) q[i]
    for (int j0 = threadIdx.x; j0 < m; j0 += 4 * blockDim.x) {
        cplx<T> acc[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] = mk<T>(0, 0);
        int i = 0;
        for (; i + 4 <= l; i += 4) {
            cplx<T> a[4][4];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int j = j0 + c * blockDim.x;
                    a[rr][c] = j < m ? A[(long)(i + rr) * m + j] : mk<T>(0, 0);
                }
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                const cplx<T> qv = q[i + rr];
#pragma unroll
                for (int c = 0; c < 4; ++c) cfmac(acc[c], a[rr][c], qv);
            }
        }
        for (; i < l; ++i) {
            const cplx<T> qv = q[i];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = j0 + c * blockDim.x;
                if (j < m) cfmac(acc[c], A[(long)i * m + j], qv);
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = j0 + c * blockDim.x;
            if (j < m) u[j] = acc[c];
        }
    }
}

template <typename T>
__device__ void mv_n(const cplx<T>* __restrict__ A, int l, int m, const cplx<T>* w, cplx<T>* u) {
    // u[i] = sum_j A[i][j] w[j]; one warp per row, two rows at a time
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp * 2; i < l; i += 2 * nw) {
        cplx<T> a0 = mk<T>(0, 0), a1 = mk<T>(0, 0);
        const bool two = (i + 1) < l;
        for (int j = lane; j < m; j += 32) {
            const cplx<T> wv = w[j];
            cfma(a0, A[(long)i * m + j], wv);
            if (two) cfma(a1, A[(long)(i + 1) * m + j], wv);
        }
        a0.x = warp_sum(a0.x);
        a0.y = warp_sum(a0.y);
        a1.x = warp_sum(a1.x);
        a1.y = warp_sum(a1.y);
        if (lane == 0) {
            u[i] = a0;
            if (two) u[i + 1] = a1;
        }
    }
}

// Normalize (per slice): scales u (length L, shared) to unit length and
// returns ||u|| in the working precision; a zero vector stays zero (its norm,
// 0, is the breakdown coefficient).  Squares are summed in the working
// precision; one thread forms the norm and its reciprocal, so no other thread
// executes float64 instructions (on GB300 one float64 instruction costs as
// much issue time as 64 float32 ones).  Only when the reciprocal is not finite
// for a positive sum (a sum too small for 1/sqrt in the working precision)
// does the scaling go through float64.
template <typename T> struct NormBc {
    double invd;
    T nrm, inv;
    int mode;
};

template <typename T>
__device__ T normalize_vec(cplx<T>* u, int L, double* red, NormBc<T>* nb) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T p = 0;
    for (int e = threadIdx.x; e < L; e += blockDim.x) p += cabs2(u[e]);
    p = warp_sum(p);
    T* redt = (T*)red;
    __syncthreads();
    if (lane == 0) redt[warp] = p;
    __syncthreads();
    if (warp == 0) {
        T t = lane < nw ? redt[lane] : (T)0;
        t = warp_sum(t);
        if (lane == 0) {
            const T inv = t > (T)0 ? (T)1 / sqrt(t) : (T)0;
            nb->nrm = sqrt(t);
            nb->inv = inv;
            nb->mode = (t > (T)0 && !isfinite(inv)) ? 1 : 0;
            if (nb->mode) nb->invd = 1.0 / sqrt((double)t);
        }
    }
    __syncthreads();
    const T nrm = nb->nrm;
    if (nb->mode == 0) {
        const T inv = nb->inv;
        for (int e = threadIdx.x; e < L; e += blockDim.x) u[e] = cscale(u[e], inv);
    } else {
        const double inv = nb->invd;
        for (int e = threadIdx.x; e < L; e += blockDim.x) {
            const cplx<T> v = u[e];
            u[e] = mk<T>((T)((double)v.x * inv), (T)((double)v.y * inv));
        }
    }
    __syncthreads();
    return nrm;
}

// ---- streaming matrix-vector products over one Fourier slice --------------
// 16-byte vector loads straight from global memory (the slice is contiguous),
// eight rows in flight per thread, one CTA barrier per product.

// u = A^H q - z * w.  Requires m / VW <= blockDim (one vector column per
// thread); rg = blockDim / (m / VW) row groups; part holds blockDim * VW entries.
template <typename T>
__device__ void mv_h_vec(const cplx<T>* __restrict__ A, int l, int m, const cplx<T>* q, const cplx<T>* w, T z,
                         cplx<T>* u, cplx<T>* part) {
    typedef cplx<T> V;
    typedef typename Vec16<T>::type LV;
    constexpr int VW = Vec16<T>::VW, UR = 8;
    const int NT = blockDim.x, tid = threadIdx.x;
    const int mv = m / VW, rg = NT / mv;
    const int g = tid / mv, cv = tid - g * mv;
    const LV* Av = (const LV*)A + cv;
    V acc[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[v] = mk<T>(0, 0);
    if (g < rg) {
        int i = g;
        for (; i + (UR - 1) * rg < l; i += UR * rg) {
            LV a[UR];
#pragma unroll
            for (int rr = 0; rr < UR; ++rr) a[rr] = __ldcg(Av + (long)(i + rr * rg) * mv);
#pragma unroll
            for (int rr = 0; rr < UR; ++rr) {
                const V qv = q[i + rr * rg];
                V e[VW];
                unpack<T>(a[rr], e);
#pragma unroll
                for (int v = 0; v < VW; ++v) cfmac(acc[v], e[v], qv);
            }
        }
        for (; i < l; i += rg) {
            const V qv = q[i];
            V e[VW];
            unpack<T>(__ldcg(Av + (long)i * mv), e);
#pragma unroll
            for (int v = 0; v < VW; ++v) cfmac(acc[v], e[v], qv);
        }
#pragma unroll
        for (int v = 0; v < VW; ++v) part[g * m + cv * VW + v] = acc[v];
    }
    __syncthreads();
    for (int j = tid; j < m; j += NT) {
        V t = mk<T>(0, 0);
        for (int p = 0; p < rg; ++p) t = cadd(t, part[p * m + j]);
        u[j] = csub(t, cscale(w[j], z));
    }
    __syncthreads();
}

// u = A w - c * q.  A warp takes RB = 4 consecutive rows, each lane a set of
// vector columns; the lanes accumulate partial sums of the four rows and one
// reduce-scatter at the end gives lane j*8 the sum of row j.
template <typename T>
__device__ void mv_n_vec(const cplx<T>* __restrict__ A, int l, int m, const cplx<T>* w, const cplx<T>* q, T cq,
                         cplx<T>* u) {
    typedef cplx<T> V;
    typedef typename Vec16<T>::type LV;
    constexpr int VW = Vec16<T>::VW, RB = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int mv = m / VW;
    const LV* Av = (const LV*)A;
    for (int i0 = warp * RB; i0 < l; i0 += nw * RB) {
        V acc[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] = mk<T>(0, 0);
#pragma unroll 2
        for (int cv = lane; cv < mv; cv += 32) {  // two iterations' loads in flight
            V wv[VW];
#pragma unroll
            for (int v = 0; v < VW; ++v) wv[v] = w[cv * VW + v];
            LV a[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (i0 + r < l) a[r] = __ldcg(Av + (long)(i0 + r) * mv + cv);
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                if (i0 + r < l) {
                    V e[VW];
                    unpack<T>(a[r], e);
#pragma unroll
                    for (int v = 0; v < VW; ++v) cfma(acc[r], e[v], wv[v]);
                }
            }
        }
        const V sum = warp_reduce_scatter<V, RB>(acc);
        const int i = i0 + (lane >> 3);
        if ((lane & 7) == 0 && i < l) u[i] = csub(sum, cscale(q[i], cq));
    }
    __syncthreads();
}

// Two classical Gram-Schmidt passes of u (length L, shared) against cnt basis
// vectors of stride L: the first kc live in shared memory (sb), the rest in
// global memory (gb).  Loads of each phase are unrolled so that many are in
// flight.  part: 4*L scratch.
template <typename T>
__device__ __forceinline__ const cplx<T>* bvec(const cplx<T>* sb, const cplx<T>* gb, int kc, int i, int L) {
    return (i < kc ? sb : gb) + (long)i * L;
}

template <typename T>
__device__ decltype(cplx<T>().x) reorth2(cplx<T>* u, const cplx<T>* sb, const cplx<T>* __restrict__ gb, int kc,
                                         int cnt, int L, cplx<T>* cf, cplx<T>* part) {
    // Returns this thread's partial sum of |u_e|^2 over its entries
    // e = threadIdx.x + j blockDim.x of the result (for normalize_into); the
    // last update is not followed by a barrier.
    typedef cplx<T> V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5, NT = blockDim.x;
    if (cnt <= 0) {
        T p = 0;
        for (int e = threadIdx.x; e < L; e += NT) p += cabs2(u[e]);
        return p;
    }
    T p = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = warp; i < cnt; i += nw) {
            const V* bv = bvec<T>(sb, gb, kc, i, L);
            V acc = mk<T>(0, 0);
            int e = lane;
            for (; e + 96 < L; e += 128) {
                const V b0 = bv[e], b1 = bv[e + 32], b2 = bv[e + 64], b3 = bv[e + 96];
                cfmac(acc, b0, u[e]);
                cfmac(acc, b1, u[e + 32]);
                cfmac(acc, b2, u[e + 64]);
                cfmac(acc, b3, u[e + 96]);
            }
            for (; e < L; e += 32) cfmac(acc, bv[e], u[e]);
            acc.x = warp_sum(acc.x);
            acc.y = warp_sum(acc.y);
            if (lane == 0) cf[i] = acc;
        }
        __syncthreads();
        // u -= sum_i basis_i cf_i, the basis split over G groups of threads
        const int G = (NT / L) >= 4 ? 4 : ((NT / L) >= 2 ? 2 : 1);
        for (int idx = threadIdx.x; idx < L * G; idx += NT) {
            const int g = idx / L, e = idx - g * L;
            V acc = mk<T>(0, 0);
            int i = g;
            for (; i + 3 * G < cnt; i += 4 * G) {
                const V b0 = bvec<T>(sb, gb, kc, i, L)[e], b1 = bvec<T>(sb, gb, kc, i + G, L)[e];
                const V b2 = bvec<T>(sb, gb, kc, i + 2 * G, L)[e], b3 = bvec<T>(sb, gb, kc, i + 3 * G, L)[e];
                cfma(acc, b0, cf[i]);
                cfma(acc, b1, cf[i + G]);
                cfma(acc, b2, cf[i + 2 * G]);
                cfma(acc, b3, cf[i + 3 * G]);
            }
            for (; i < cnt; i += G) cfma(acc, bvec<T>(sb, gb, kc, i, L)[e], cf[i]);
            part[g * L + e] = acc;
        }
        __syncthreads();
        p = 0;
        for (int e = threadIdx.x; e < L; e += NT) {
            V t = u[e];
            for (int g = 0; g < G; ++g) t = csub(t, part[g * L + e]);
            u[e] = t;
            p += cabs2(t);
        }
        if (pass == 0) __syncthreads();
    }
    return p;
}

// Normalize u (length L, shared) given each thread's partial sum of squares
// over its entries e = threadIdx.x + j blockDim.x (as reorth2 returns it):
// writes u / ||u|| to dst (shared) and, if given, dstg (global), and returns
// ||u|| in the working precision; a zero vector gives zeros and norm 0.  One
// thread forms the norm and its reciprocal (float64 only when the
// working-precision reciprocal of a positive sum is not finite).
template <typename T>
__device__ T normalize_into(const cplx<T>* u, int L, T p, double* red, NormBc<T>* nb, cplx<T>* dst,
                            cplx<T>* dstg) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    p = warp_sum(p);
    T* redt = (T*)red;
    __syncthreads();  // u complete; redt free
    if (lane == 0) redt[warp] = p;
    __syncthreads();
    if (warp == 0) {
        T t = lane < nw ? redt[lane] : (T)0;
        t = warp_sum(t);
        if (lane == 0) {
            const T inv = t > (T)0 ? (T)1 / sqrt(t) : (T)0;
            nb->nrm = sqrt(t);
            nb->inv = inv;
            nb->mode = (t > (T)0 && !isfinite(inv)) ? 1 : 0;
            if (nb->mode) nb->invd = 1.0 / sqrt((double)t);
        }
    }
    __syncthreads();
    const T nrm = nb->nrm;
    if (nb->mode == 0) {
        const T inv = nb->inv;
        for (int e = threadIdx.x; e < L; e += blockDim.x) {
            const cplx<T> v = cscale(u[e], inv);
            dst[e] = v;
            if (dstg) dstg[e] = v;
        }
    } else {
        const double inv = nb->invd;
        for (int e = threadIdx.x; e < L; e += blockDim.x) {
            const cplx<T> x = u[e];
            const cplx<T> v = mk<T>((T)((double)x.x * inv), (T)((double)x.y * inv));
            dst[e] = v;
            if (dstg) dstg[e] = v;
        }
    }
    __syncthreads();
    return nrm;
}

// Persistent tGKB.  Outputs per slice: W (k_max x m), Q (k_max+1 x l),
// c (k_max), z (k_max+1), Xhat (m) for the chosen k; State k/status; info.
template <typename T, bool VEC, int NT>
__global__ void __launch_bounds__(NT, NT >= 1024 ? 1 : (NT >= 512 ? 2 : 4))
k_gkb(const cplx<T>* __restrict__ Ahat, const cplx<T>* __restrict__ Bhat, int l, int m, int n, int h, int k_max,
      double tau_delta, cplx<T>* Wb, cplx<T>* Qb, T* cc, T* zz, double* res2, unsigned* counters,
      cplx<T>* Xhat, State* st, tp_info* info, double* res_hist, long long spin_cycles, int write_info, int kc,
      int bs, int extra) {
    // bs: column stride of Bhat and Xhat (the lateral slice count of B; the
    // pointers already point at this slice's column)
    typedef cplx<T> V;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = l > m ? l : m;
    V* q = (V*)smraw;           // l
    V* w = q + l;               // m
    V* u = w + m;               // L
    V* cf = u + L;              // k_max + 1
    V* part = cf + k_max + 1;   // max(4 L, NT * VW)
    const int part_n = (4 * L > NT * (16 / (int)sizeof(V))) ? 4 * L : NT * (16 / (int)sizeof(V));
    V* Wc = part + part_n;      // kc cached vectors of W (m each)
    V* Qc = Wc + (long)kc * m;  // kc cached vectors of Q (l each)
    __shared__ GkbShared S;
    __shared__ double red[33];
    __shared__ NormBc<T> nb;
    __shared__ T yt[GKB_KMAX];
    __shared__ int flag_done, flag_timeout;
    const int s = blockIdx.x, tid = threadIdx.x;
    const V* A = Ahat + (long)s * l * m;
    V* W = Wb + (long)s * k_max * m;
    V* Qv = Qb + (long)s * (k_max + 1) * l;
    T* cs_ = cc + (long)s * k_max;
    T* zs_ = zz + (long)s * (k_max + 1);
    const double ws = parseval_w(s, n);

    for (int e = tid; e < l; e += blockDim.x) u[e] = Bhat[((long)s * l + e) * bs];
    for (int e = tid; e < m; e += blockDim.x) w[e] = mk<T>(0, 0);
    __syncthreads();
    const T z1 = normalize_vec<T>(u, l, red, &nb);
    for (int e = tid; e < l; e += blockDim.x) {
        q[e] = u[e];
        Qv[e] = u[e];
        if (kc > 0) Qc[e] = u[e];
    }
    if (tid == 0) {
        zs_[0] = z1;
        flag_done = 0;
        flag_timeout = 0;
    }
    __syncthreads();

    const double td2n = (double)n * tau_delta * tau_delta;
    // Givens state (thread 0): phibar, previous rotation, orphan residual
    // The rotations run in the working precision: the bidiagonal entries are
    // working-precision norms, and a float64 square root and division on one
    // thread cost thousands of cycles per step on this GPU (1/64-rate float64).
    T phibar = z1, cs_prev = 1, sn_prev = 0, orphan = 0;
    T zprev = z1;
    int k = k_max;
    // Step i publishes its residual and goes on; the discrepancy test of step
    // i-1 is taken after step i's first product (which hides the grid-wide
    // wait), and a stop discards step i before it writes anything.
    for (int i = 1; i <= k_max + 1; ++i) {
        const bool step = i <= k_max;
        // W_i = A^T * Q_i - W_{i-1} * z_i
        if (step) {
            if (VEC) {
                mv_h_vec<T>(A, l, m, q, w, zprev, u, part);
            } else {
                mv_h<T>(A, l, m, q, u);
                __syncthreads();
                for (int e = tid; e < m; e += blockDim.x) u[e] = csub(u[e], cscale(w[e], zprev));
                __syncthreads();
            }
        }
        if (i >= 2) {
            if (tid == 0) {
                // wait for every slice to finish step i-1 (bounded)
                const long long t0 = clock64();
                while (ld_acquire(&counters[i - 1]) < (unsigned)(h + extra)) {
                    if (clock64() - t0 > spin_cycles) {
                        flag_timeout = 1;
                        break;
                    }
                }
            }
            __syncthreads();
            // squared residual of step i-1 (times n): the same fixed-order sum
            // over slices in every CTA; compared with n (tau delta)^2
            if (tid < 32 && !flag_timeout) {
                double tot = 0.0;
                for (int s2 = tid; s2 < h; s2 += 32) tot += __ldcg(&res2[(long)(i - 1) * h + s2]);
                tot = warp_sum(tot);
                if (tid == 0) {
                    S.res[i - 1] = tot;
                    if (tot <= td2n) flag_done = 1;
                }
            }
            __syncthreads();
            if (flag_timeout || flag_done) {
                k = i - 1;
                break;
            }
        }
        if (!step) break;
        // reorthogonalise ; Normalize -> c_i, w = W_i
        const T pw = reorth2<T>(u, Wc, W, kc, i - 1, m, cf, part);
        const T ci = normalize_into<T>(u, m, pw, red, &nb, w, W + (long)(i - 1) * m);
        if (i - 1 < kc)
            for (int e = tid; e < m; e += blockDim.x) Wc[(long)(i - 1) * m + e] = w[e];
        // Q_{i+1} = A * W_i - Q_i * c_i ; reorthogonalise ; Normalize -> z_{i+1}
        if (VEC) {
            mv_n_vec<T>(A, l, m, w, q, ci, u);
        } else {
            mv_n<T>(A, l, m, w, u);
            __syncthreads();
            for (int e = tid; e < l; e += blockDim.x) u[e] = csub(u[e], cscale(q[e], ci));
            __syncthreads();
        }
        const T pq = reorth2<T>(u, Qc, Qv, kc, i, l, cf, part);
        const T zi = normalize_into<T>(u, l, pq, red, &nb, q, Qv + (long)i * l);
        if (i < kc)
            for (int e = tid; e < l; e += blockDim.x) Qc[(long)i * l + e] = q[e];
        if (tid == 0) {
            cs_[i - 1] = ci;
            zs_[i] = zi;
            // Givens QR of the lower-bidiagonal slice: column i has c_i on the
            // diagonal, z_{i+1} below it.
            const T cid = ci, zid = zi;
            const T rhobar = (i == 1) ? cid : cs_prev * cid;
            S.theta[i - 1] = (i == 1) ? 0.0 : (double)(sn_prev * cid);   // R(i-1, i)
            const T rho = sqrt(fma(rhobar, rhobar, zid * zid));  // norms of working-precision vectors
            T c = 1, sn = 0;
            if (rho > (T)0) {
                const T irho = (T)1 / rho;
                c = rhobar * irho;
                sn = zid * irho;
                S.phi[i - 1] = (double)(c * phibar);
                phibar = -sn * phibar;
            } else {  // zero column: its right-hand side entry stays unmatched
                S.phi[i - 1] = 0.0;
                orphan += phibar * phibar;
                phibar = 0;
            }
            S.rho[i - 1] = rho;
            cs_prev = c;
            sn_prev = sn;
            res2[(long)i * h + s] = ws * (double)(orphan + phibar * phibar);
            // step i done here (release: the residual above is visible first); the test comes after the next product
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&counters[i]) : "memory");
        }
        zprev = zi;
    }
    // back substitution R y = phi (rho on the diagonal, theta above it); the
    // residuals from their squares (times n)
    if (tid == 0) {
        for (int j = 1; j <= k; ++j) S.res[j] = sqrt(S.res[j] / (double)n);
        for (int j = k - 1; j >= 0; --j) {
            double v = S.phi[j];
            if (j + 1 < k) v -= S.theta[j + 1] * S.y[j + 1];
            S.y[j] = S.rho[j] > 0.0 ? v / S.rho[j] : 0.0;
            yt[j] = (T)S.y[j];
        }
    }
    __syncthreads();
    // X-hat = W y in the working precision
    for (int e = tid; e < m; e += blockDim.x) {
        V x = mk<T>(0, 0);
        for (int j = 0; j < k; ++j) {
            const V v = W[(long)j * m + e];
            x.x = fma(v.x, yt[j], x.x);
            x.y = fma(v.y, yt[j], x.y);
        }
        Xhat[((long)s * m + e) * bs] = x;
    }
    if (s == 0 && tid == 0) {
        int status = flag_timeout ? TP_ERR_TIMEOUT : (flag_done ? TP_OK : TP_ERR_NOT_CONVERGED);
        st->k = k;
        st->status = status;
        const double res_k = flag_timeout ? -1.0 : S.res[k];
        double margin = fabs(res_k - tau_delta) / tau_delta;
        if (k >= 2) margin = fmin(margin, fabs(S.res[k - 1] - tau_delta) / tau_delta);
        if (res_hist) {
            res_hist[0] = -1.0;
            for (int j = 1; j <= k_max; ++j) res_hist[j] = j <= k ? S.res[j] : -1.0;
        }
        if (write_info) {
            tp_info o;
            o.status = status;
            o.k = k;
            o.r = k;
            o.sweeps = 0;
            o.residual = res_k;
            o.tau_delta = tau_delta;
            o.eta = 0.0;
            o.mu = 0.0;
            o.margin = margin;
            o.norm_a2 = 0.0;
            *info = o;
        }
    }
}

// ---------------------------------------------------------------------------
// nested_tGKB_p (Algorithm 6): one Krylov basis, grown by Algorithm 4 from the
// first lateral slice, serves the p slices in turn.  Slice j's projected
// problem min ||P_k y - Q_{k+1}^H b_j|| is solved with the Givens QR of the
// common bidiagonal P_k: the rotation of every step is kept (per Fourier
// slice), the current slice's right-hand side coefficients are rotated as the
// basis grows, and the next slice replays the stored rotations on its own
// coefficients.  Tests are not lagged: after each published residual every
// CTA waits (bounded) for all Fourier slices, then all take the same
// decision.  Events (a residual after a step, a new slice's first residual)
// index the counters.
struct GknArgs {
    const void* Ahat;
    const void* Bhat;     // (h, l, p)
    void* Wb;             // (h, k_max, m)
    void* Qb;             // (h, k_max+1, l)
    void* Xhat;           // (h, m, p)
    double* phi;          // (h, k_max, 2): rotated right-hand side of the current slice
    double* rot;          // (h, k_max, 3): cs, sn, rho of each step's rotation
    double* res2;         // (k_max + p + 1, h)
    unsigned* counters;   // k_max + p + 1, zeroed by the launcher
    const double* td;     // p values eta * delta_j (device)
    tp_info* info;        // p records
    double* res_hist;     // optional (p, k_max+1)
    long long spin;
    int extra;            // arrivals awaited beyond the grid (0; 1 under tp_wait_stall)
    int l, m, n, h, k_max, p, k_init;
};

struct GknShared {
    double theta[GKB_KMAX + 1];
    double cs_prev, sn_prev, orphan, res_prev, tot;
    double2 phibar;
    int k, j, e, timeout, have_prev;
};

// Complex dot q^H b over the CTA (working precision per thread and warp,
// float64 across warps); every thread gets the result.  red: 64 doubles.
template <typename T>
__device__ double2 block_dot(const cplx<T>* q, const cplx<T>* b, int L, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    cplx<T> acc = mk<T>(0, 0);
    for (int e = threadIdx.x; e < L; e += blockDim.x) cfmac(acc, q[e], b[e]);
    acc.x = warp_sum(acc.x);
    acc.y = warp_sum(acc.y);
    __syncthreads();
    if (lane == 0) {
        red[warp] = (double)acc.x;
        red[32 + warp] = (double)acc.y;
    }
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    for (int i = 0; i < nw; ++i) {
        r.x += red[i];
        r.y += red[32 + i];
    }
    __syncthreads();
    return r;
}

template <typename T, bool VEC, int NT>
__global__ void __launch_bounds__(NT, NT >= 1024 ? 1 : (NT >= 512 ? 2 : 4)) k_gkb_nested(const GknArgs a) {
    typedef cplx<T> V;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int l = a.l, m = a.m, n = a.n, h = a.h, k_max = a.k_max, p = a.p;
    const int L = l > m ? l : m;
    V* q = (V*)smraw;           // l
    V* w = q + l;               // m
    V* u = w + m;               // L
    V* bj = u + L;              // l: the current lateral slice
    V* cf = bj + l;             // k_max + 1
    V* part = cf + k_max + 1;   // max(4 L, NT * VW)
    __shared__ GknShared S;
    __shared__ double red[64];
    __shared__ NormBc<T> nb;
    __shared__ V yt[GKB_KMAX];
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NT / 32;
    const V* A = (const V*)a.Ahat + (long)s * l * m;
    const V* Bh = (const V*)a.Bhat;
    V* W = (V*)a.Wb + (long)s * k_max * m;
    V* Qv = (V*)a.Qb + (long)s * (k_max + 1) * l;
    V* Xh = (V*)a.Xhat;
    double* phi = a.phi + (long)s * k_max * 2;
    double* rot = a.rot + (long)s * k_max * 3;
    const double ws = parseval_w(s, n);
    const int k_first = a.k_init < k_max ? a.k_init : k_max;

    for (int e = tid; e < l; e += NT) {
        const V b = Bh[((long)s * l + e) * p];
        u[e] = b;
        bj[e] = b;
    }
    for (int e = tid; e < m; e += NT) w[e] = mk<T>(0, 0);
    if (s == 0 && a.res_hist)
        for (int e = tid; e < p * (k_max + 1); e += NT) a.res_hist[e] = -1.0;
    __syncthreads();
    const T z1 = normalize_vec<T>(u, l, red, &nb);
    for (int e = tid; e < l; e += NT) {
        q[e] = u[e];
        Qv[e] = u[e];
    }
    if (tid == 0) {
        S.cs_prev = 1.0;
        S.sn_prev = 0.0;
        S.orphan = 0.0;
        S.phibar = make_double2((double)z1, 0.0);  // q_1^H b_1 = z_1
        S.k = 0;
        S.j = 0;
        S.e = 0;
        S.timeout = 0;
        S.have_prev = 0;
    }
    __syncthreads();
    T zprev = z1;

    for (;;) {
        if (S.k < k_max) {
            // one more step of Algorithm 4: W_i, c_i, Q_{i+1}, z_{i+1}
            const int i = S.k + 1;
            if (VEC) {
                mv_h_vec<T>(A, l, m, q, w, zprev, u, part);
            } else {
                mv_h<T>(A, l, m, q, u);
                __syncthreads();
                for (int e = tid; e < m; e += NT) u[e] = csub(u[e], cscale(w[e], zprev));
                __syncthreads();
            }
            const T pw = reorth2<T>(u, nullptr, W, 0, i - 1, m, cf, part);
            const T ci = normalize_into<T>(u, m, pw, red, &nb, w, W + (long)(i - 1) * m);
            if (VEC) {
                mv_n_vec<T>(A, l, m, w, q, ci, u);
            } else {
                mv_n<T>(A, l, m, w, u);
                __syncthreads();
                for (int e = tid; e < l; e += NT) u[e] = csub(u[e], cscale(q[e], ci));
                __syncthreads();
            }
            const T pq = reorth2<T>(u, nullptr, Qv, 0, i, l, cf, part);
            const T zi = normalize_into<T>(u, l, pq, red, &nb, q, Qv + (long)i * l);
            const double2 cn = block_dot<T>(q, bj, l, red);  // q_{i+1}^H b_j
            if (tid == 0) {
                // Givens QR of column i of the bidiagonal (c_i on the diagonal,
                // z_{i+1} below), applied to the current right-hand side
                const double cid = ci, zid = zi;
                const double rhobar = (i == 1) ? cid : S.cs_prev * cid;
                S.theta[i - 1] = (i == 1) ? 0.0 : S.sn_prev * cid;  // R(i-1, i)
                const double rho = givens_norm<T>(rhobar, zid);
                double c = 1.0, sn = 0.0;
                const double2 pb = S.phibar;
                if (rho > 0.0) {
                    const double irho = 1.0 / rho;
                    c = rhobar * irho;
                    sn = zid * irho;
                    phi[2 * (i - 1)] = c * pb.x + sn * cn.x;
                    phi[2 * (i - 1) + 1] = c * pb.y + sn * cn.y;
                    S.phibar = make_double2(-sn * pb.x + c * cn.x, -sn * pb.y + c * cn.y);
                } else {  // zero column: its right-hand side entry stays unmatched
                    phi[2 * (i - 1)] = 0.0;
                    phi[2 * (i - 1) + 1] = 0.0;
                    S.orphan += pb.x * pb.x + pb.y * pb.y;
                    S.phibar = cn;
                }
                rot[3 * (i - 1)] = c;
                rot[3 * (i - 1) + 1] = sn;
                rot[3 * (i - 1) + 2] = rho;
                S.cs_prev = c;
                S.sn_prev = sn;
                S.k = i;
            }
            zprev = zi;
            __syncthreads();
        }
        const int kk = S.k;
        if (kk < k_first) continue;
        bool finished = false;
        // the test of the current slice at this k, then of every following
        // slice that the present basis already satisfies
        for (;;) {
            if (tid == 0) {
                const double2 pb = S.phibar;
                a.res2[(long)S.e * h + s] = ws * (S.orphan + pb.x * pb.x + pb.y * pb.y);
                asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&a.counters[S.e]) : "memory");
                const long long t0 = clock64();
                while (ld_acquire(&a.counters[S.e]) < (unsigned)(h + a.extra)) {
                    if (clock64() - t0 > a.spin) {
                        S.timeout = 1;
                        break;
                    }
                }
            }
            __syncthreads();
            if (warp == 0) {  // the same fixed-order sum in every CTA
                double tot = 0.0;
                if (!S.timeout)
                    for (int s2 = lane; s2 < h; s2 += 32) tot += __ldcg(&a.res2[(long)S.e * h + s2]);
                tot = warp_sum(tot);
                if (lane == 0) {
                    S.tot = tot;
                    ++S.e;
                }
            }
            __syncthreads();
            const int j = S.j;
            const double tdj = a.td[j], tot = S.tot;
            const bool met = !S.timeout && tot < (double)n * tdj * tdj;
            if (s == 0 && tid == 0 && a.res_hist && !S.timeout) a.res_hist[(long)j * (k_max + 1) + kk] = sqrt(tot / n);
            if (!met && !S.timeout && kk < k_max) {
                if (tid == 0) {
                    S.res_prev = tot;
                    S.have_prev = 1;
                }
                __syncthreads();
                break;  // extend the basis
            }
            // accept slice j at k = kk: back substitution R y = phi (complex
            // right-hand side), then X-hat_j = W_k y
            if (tid == 0) {
                double2 yn = make_double2(0.0, 0.0);
                for (int t = kk - 1; t >= 0; --t) {
                    double vx = phi[2 * t], vy = phi[2 * t + 1];
                    if (t + 1 < kk) {
                        vx -= S.theta[t + 1] * yn.x;
                        vy -= S.theta[t + 1] * yn.y;
                    }
                    const double rho = rot[3 * t + 2];
                    yn = rho > 0.0 ? make_double2(vx / rho, vy / rho) : make_double2(0.0, 0.0);
                    yt[t] = mk<T>((T)yn.x, (T)yn.y);
                }
            }
            __syncthreads();
            for (int e = tid; e < m; e += NT) {
                V x = mk<T>(0, 0);
                for (int t = 0; t < kk; ++t) cfma(x, W[(long)t * m + e], yt[t]);
                Xh[((long)s * m + e) * p + j] = x;
            }
            if (s == 0 && tid == 0) {
                const int status = S.timeout ? TP_ERR_TIMEOUT : (met ? TP_OK : TP_ERR_NOT_CONVERGED);
                const double res_k = S.timeout ? -1.0 : sqrt(tot / n);
                double margin = fabs(res_k - tdj) / tdj;
                if (S.have_prev && !S.timeout) margin = fmin(margin, fabs(sqrt(S.res_prev / n) - tdj) / tdj);
                tp_info o;
                o.status = status;
                o.k = kk;
                o.r = kk;
                o.sweeps = 0;
                o.residual = res_k;
                o.tau_delta = tdj;
                o.eta = 0.0;
                o.mu = 0.0;
                o.margin = margin;
                o.norm_a2 = 0.0;
                a.info[j] = o;
            }
            __syncthreads();
            if (j + 1 == p || S.timeout) {
                if (S.timeout) {  // the slices not reached: zero solutions, status TIMEOUT
                    for (int jj = j + 1; jj < p; ++jj) {
                        for (int e = tid; e < m; e += NT) Xh[((long)s * m + e) * p + jj] = mk<T>(0, 0);
                        if (s == 0 && tid == 0) {
                            tp_info o = {};
                            o.status = TP_ERR_TIMEOUT;
                            o.k = kk;
                            o.r = kk;
                            o.residual = -1.0;
                            o.tau_delta = a.td[jj];
                            a.info[jj] = o;
                        }
                    }
                }
                finished = true;
                break;
            }
            // next slice: its coefficients against Q_{k+1}, rotated by the
            // stored rotations of steps 1..k
            for (int e = tid; e < l; e += NT) bj[e] = Bh[((long)s * l + e) * p + j + 1];
            __syncthreads();
            for (int t = warp; t <= kk; t += nw) {
                const V* qt = Qv + (long)t * l;
                V acc = mk<T>(0, 0);
                for (int e = lane; e < l; e += 32) cfmac(acc, __ldcg(qt + e), bj[e]);
                acc.x = warp_sum(acc.x);
                acc.y = warp_sum(acc.y);
                if (lane == 0) cf[t] = acc;
            }
            __syncthreads();
            if (tid == 0) {
                double2 pb = make_double2((double)cf[0].x, (double)cf[0].y);
                double orphan = 0.0;
                for (int t = 0; t < kk; ++t) {
                    const double c = rot[3 * t], sn = rot[3 * t + 1], rho = rot[3 * t + 2];
                    const double2 cn = make_double2((double)cf[t + 1].x, (double)cf[t + 1].y);
                    if (rho > 0.0) {
                        phi[2 * t] = c * pb.x + sn * cn.x;
                        phi[2 * t + 1] = c * pb.y + sn * cn.y;
                        pb = make_double2(-sn * pb.x + c * cn.x, -sn * pb.y + c * cn.y);
                    } else {
                        phi[2 * t] = 0.0;
                        phi[2 * t + 1] = 0.0;
                        orphan += pb.x * pb.x + pb.y * pb.y;
                        pb = cn;
                    }
                }
                S.phibar = pb;
                S.orphan = orphan;
                S.j = j + 1;
                S.have_prev = 0;
            }
            __syncthreads();
        }
        if (finished) break;
    }
}

// ---------------------------------------------------------------------------
// Tikhonov on the projected problem of each slice:
//   min ||P y - z1 e1||^2 + lam^2 ||y||^2,  lam^2 = 1/mu,
// solved by Givens QR of [P; lam I] (two rotations per column); returns the
// data residual ||P y - z1 e1||^2 and optionally y.
// ---------------------------------------------------------------------------
template <typename R>
__device__ R damped_bidiag(const R* c, const R* z, int k, R lam, R* y, R* scr, int kcap, int stride) {
    // scr: per-thread scratch of 4 arrays (rho, theta, phi, y) of kcap entries,
    // entry j of an array at scr[j * stride] (stride = threads sharing the
    // buffer, so that neighbouring threads touch neighbouring addresses).
    // Working precision R: the bidiagonal entries come from R-precision vectors.
    struct Strided {
        R* p;
        int st;
        __device__ R& operator[](int j) const { return p[(long)j * st]; }
    };
    const long a = (long)kcap * stride;
    Strided rho{scr, stride}, theta{scr + a, stride}, phi{scr + 2 * a, stride};
    Strided yy = y ? Strided{y, 1} : Strided{scr + 3 * a, stride};
    R rhobar = k > 0 ? c[0] : (R)0, phibar = z[0];
    for (int j = 0; j < k; ++j) {
        const R rh = hypot(rhobar, lam);          // eliminate the damping row
        const R c1 = rh > (R)0 ? rhobar / rh : (R)1;
        const R ph = c1 * phibar;
        const R zj = z[j + 1];
        const R rj = hypot(rh, zj);               // eliminate z_{j+2}
        R cs = 1, sn = 0;
        if (rj > (R)0) {
            cs = rh / rj;
            sn = zj / rj;
        }
        rho[j] = rj;
        phi[j] = cs * ph;
        phibar = -sn * ph;
        if (j + 1 < k) {
            theta[j + 1] = sn * c[j + 1];
            rhobar = cs * c[j + 1];
        }
    }
    for (int j = k - 1; j >= 0; --j) {
        R v = phi[j];
        if (j + 1 < k) v -= theta[j + 1] * yy[j + 1];
        yy[j] = rho[j] > (R)0 ? v / rho[j] : (R)0;
    }
    // data residual: r_1 = c_1 y_1 - z_1, r_j = z_j y_{j-1} + c_j y_j, r_{k+1} = z_{k+1} y_k
    R r2 = 0;
    for (int j = 0; j <= k; ++j) {
        R v = (j < k ? c[j] * yy[j] : (R)0) + (j > 0 ? z[j] * yy[j - 1] : (R)0);
        if (j == 0) v -= z[0];
        r2 = fma(v, v, r2);
    }
    return r2;
}

struct TikState {
    double lo, hi, t;
    int done, status, round;
    unsigned arrived;
};

constexpr int TIK_P = 256;
// lam_p = 10^(-t_p / 2) at the TIK_P points t_p = lo + (hi - lo) p / (TIK_P - 1)
// of the current bracket, each thread its own point: x = -t_p log2(10) / 2 in
// float64, split as x = e + f (e an integer, 0 <= f < 1), lam = 2^f 2^e with
// 2^f in the working precision (a relative error of a few units in its last
// place, the precision lam is used in).  All TIK_P threads call it.
template <typename R> __device__ __forceinline__ R exp2_split(double x);
template <> __device__ __forceinline__ float exp2_split<float>(double x) {
    const double e = floor(x);
    return ldexpf(exp2f((float)(x - e)), (int)e);
}
template <> __device__ __forceinline__ double exp2_split<double>(double x) { return exp2(x); }

template <typename R>
__device__ void fill_lam(const TikState* ts, R* lam) {
    const int p = threadIdx.x;
    const double lo = ts->lo, hi = ts->hi;
    const double t = p == TIK_P - 1 ? hi : lo + (hi - lo) * ((double)p * (1.0 / (TIK_P - 1)));
    lam[p] = exp2_split<R>(-1.66096404744368117393 * t);  // -log2(10) / 2
}

// New bracket from the residuals at the TIK_P points (one CTA of TIK_P
// threads): the first point whose residual is at most tau*delta closes it.
// The slice sum runs in a fixed order with Kahan compensation in the working
// precision; "above" means sum/n > (tau delta)^2, i.e. residual > tau*delta.
template <typename R>
__device__ void tik_select(const R* out, int h, R thr, double log_tol, TikState* ts, R* lamv) {
    __shared__ unsigned char above[TIK_P];
    const int p = threadIdx.x;
    R a = 0, comp = 0;
    constexpr int SB = 16;  // slice values loaded ahead of the (ordered) Kahan additions
    for (int s0 = 0; s0 < h; s0 += SB) {
        R v[SB];
#pragma unroll
        for (int u = 0; u < SB; ++u) v[u] = s0 + u < h ? __ldcg(&out[(long)(s0 + u) * TIK_P + p]) : (R)0;
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            if (s0 + u >= h) break;
            const R y = v[u] - comp;
            const R t = a + y;
            comp = (t - a) - y;
            a = t;
        }
    }
    above[p] = a > thr ? 1 : 0;
    __syncthreads();
    if (p == 0) {
        const double lo = ts->lo, hi = ts->hi;
        bool fin = false;
        if (ts->round == 0) {
            if (above[TIK_P - 1]) {  // even mu_hi leaves the residual above tau*delta
                ts->t = hi;
                ts->status = TP_ERR_NOT_CONVERGED;
                fin = true;
            } else if (!above[0]) {
                ts->t = lo;
                fin = true;
            }
        }
        if (!fin) {
            int ps = TIK_P - 1;
            for (int i = 1; i < TIK_P; ++i)
                if (!above[i]) {
                    ps = i;
                    break;
                }
            auto pt = [&](int i) {
                return i == 0 ? lo : (i == TIK_P - 1 ? hi : lo + (hi - lo) * (double)i / (double)(TIK_P - 1));
            };
            ts->lo = pt(ps - 1);
            ts->hi = pt(ps);
            ts->round += 1;
            if (ts->hi - ts->lo <= log_tol) {
                ts->t = ts->hi;
                fin = true;
            }
        }
        ts->done = fin ? 1 : 0;
        ts->arrived = 0;
    }
    __syncthreads();
    if (!ts->done) fill_lam<R>(ts, lamv);
}

// The data residual ||P y - z_1 e_1||^2 of the damped problem, as
// damped_bidiag computes it, with the Givens data of the forward sweep in
// shared memory (entry j of thread p at [j * TIK_P + p]) and the residual
// entries formed during the back substitution (y is not stored).
template <typename R>
__device__ R damped_resid_smem(const R* c, const R* z, int k, R lam, R* rho, R* theta, R* phi) {
    const int p = threadIdx.x;
    R rhobar = k > 0 ? c[0] : (R)0, phibar = z[0];
    for (int j = 0; j < k; ++j) {
        const R rh = sqrt(fma(rhobar, rhobar, lam * lam));  // eliminate the damping row
        const R c1 = rh > (R)0 ? rhobar / rh : (R)1;
        const R ph = c1 * phibar;
        const R zj = z[j + 1];
        const R rj = sqrt(fma(rh, rh, zj * zj));           // eliminate z_{j+2}
        R cs = 1, sn = 0;
        if (rj > (R)0) {
            const R ir = (R)1 / rj;
            cs = rh * ir;
            sn = zj * ir;
        }
        rho[j * TIK_P + p] = rj;
        phi[j * TIK_P + p] = cs * ph;
        phibar = -sn * ph;
        if (j + 1 < k) {
            theta[(j + 1) * TIK_P + p] = sn * c[j + 1];
            rhobar = cs * c[j + 1];
        }
    }
    // back substitution; residual entries r_k = z_k y_{k-1},
    // r_j = z_j y_{j-1} + c_j y_j, r_0 = c_0 y_0 - z_0
    R r2 = 0, ynext = 0;
    for (int j = k - 1; j >= 0; --j) {
        R v = phi[j * TIK_P + p];
        if (j + 1 < k) v -= theta[(j + 1) * TIK_P + p] * ynext;
        const R rr = rho[j * TIK_P + p];
        const R y = rr > (R)0 ? v / rr : (R)0;
        const R e = z[j + 1] * y + (j + 1 < k ? c[j + 1] * ynext : (R)0);
        r2 = fma(e, e, r2);
        ynext = y;
    }
    const R e0 = (k > 0 ? c[0] * ynext : (R)0) - z[0];
    return fma(e0, e0, r2);
}

// Largest k whose Givens data fit in the round kernel's shared memory.
template <typename R> constexpr int tik_smem_k() { return (int)(160 * 1024 / (3 * TIK_P * sizeof(R))); }

// One multisection round: the data residual at the TIK_P points of the
// bracket for every slice (out[s*TIK_P + p]); the last CTA to finish selects
// the next bracket.
template <typename R>
__global__ void __launch_bounds__(TIK_P)
k_tik_round(const R* cc, const R* zz, int k_max, const State* st, TikState* ts, R* lamv, int h, int n, R* out,
            R* scratch, R thr, double log_tol) {
    if (ts->done) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int last;
    const int s = blockIdx.x, p = threadIdx.x, k = st->k;
    const R lam = lamv[p];
    R r2;
    if (k <= tik_smem_k<R>()) {
        R* sm = (R*)smraw;
        r2 = damped_resid_smem<R>(cc + (long)s * k_max, zz + (long)s * (k_max + 1), k, lam, sm, sm + k * TIK_P,
                                  sm + 2 * k * TIK_P);
    } else {
        R* scr = scratch + (long)s * TIK_P * 4 * k_max + p;
        r2 = damped_bidiag<R>(cc + (long)s * k_max, zz + (long)s * (k_max + 1), k, lam, nullptr, scr, k_max,
                              TIK_P);
    }
    out[(long)s * TIK_P + p] = ((s == 0 || 2 * s == n) ? (R)1 : (R)2) * r2;
    __threadfence();
    __syncthreads();
    if (p == 0) last = atomicAdd(&ts->arrived, 1u) == (unsigned)(h - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    tik_select<R>(out, h, thr, log_tol, ts, lamv);
}

// final: y_mu per slice, Xhat = W y, residual; info
template <typename T>
__global__ void __launch_bounds__(256)
k_tik_final(const T* cc, const T* zz, int k_max, const cplx<T>* Wb, int m, const State* st,
            const TikState* ts, int n, double* fout, cplx<T>* Xhat, T* scratch) {
    __shared__ T y[GKB_KMAX];
    const int s = blockIdx.x, k = st->k;
    if (threadIdx.x == 0) {
        const T lam = (T)pow(10.0, -0.5 * ts->t);
        const T r2 = damped_bidiag<T>(cc + (long)s * k_max, zz + (long)s * (k_max + 1), k, lam, y,
                                      scratch + (long)s * TIK_P * 4 * k_max, k_max, 1);
        fout[s] = parseval_w(s, n) * (double)r2;
    }
    __syncthreads();
    const cplx<T>* W = Wb + (long)s * k_max * m;
    for (int e = threadIdx.x; e < m; e += blockDim.x) {
        cplx<T> x = mk<T>(0, 0);
        for (int j = 0; j < k; ++j) {
            const cplx<T> v = W[(long)j * m + e];
            x.x = fma(v.x, y[j], x.x);
            x.y = fma(v.y, y[j], x.y);
        }
        Xhat[(long)s * m + e] = x;
    }
}

__global__ void k_tik_info(const double* fout, int h, int n, const State* st, const TikState* ts, double tau_delta,
                           tp_info* info) {
    double a = 0.0;  // lanes take every 32nd slice, then a fixed-order warp sum
    for (int s = threadIdx.x; s < h; s += 32) a += fout[s];
    a = warp_sum(a);
    if (threadIdx.x != 0) return;
    tp_info o;
    o.status = st->status == TP_ERR_TIMEOUT ? TP_ERR_TIMEOUT : ts->status;
    o.k = st->k;
    o.r = st->k;
    o.sweeps = ts->round;
    o.residual = sqrt(a / (double)n);
    o.tau_delta = tau_delta;
    o.eta = 0.0;
    o.mu = pow(10.0, ts->t);
    o.margin = fabs(o.residual - tau_delta) / tau_delta;
    o.norm_a2 = 0.0;
    *info = o;
}

template <typename R>
__global__ void __launch_bounds__(TIK_P) k_tik_init(TikState* ts, R* lamv, double lo, double hi) {
    if (threadIdx.x == 0) {
        ts->lo = lo;
        ts->hi = hi;
        ts->t = hi;
        ts->done = 0;
        ts->status = TP_OK;
        ts->round = 0;
        ts->arrived = 0;
    }
    __syncthreads();
    fill_lam<R>(ts, lamv);
}

// ---------------------------------------------------------------------------
template <typename T>
struct GkWs {
    State* st;
    TikState* ts;
    unsigned* counters;
    double *res2, *fout;
    T *cc, *zz, *tout, *lam, *tscr;
    double* gv;  // Givens data of the batched kernel (p > 1)
    double *partsA, *partsB;  // squared-norm partials of the DFTs of A and B (non-finite input check)
    int nA, nB;
    cplx<T> *Ahat, *Bhat, *W, *Q, *Xhat;
    size_t bytes;
};

template <typename T>
static GkWs<T> gk_carve(void* base, int l, int m, int n, int k_max, int p) {
    // p > 1: bases and step residuals for one group of GKM_PB lateral slices
    // (groups run one after another), B-hat and X-hat for all p
    typedef cplx<T> V;
    const long h = n / 2 + 1;
    const long pb = p > 1 ? GKM_PB : 1;
    Carver c(base, 0);
    GkWs<T> w;
    w.st = c.take<State>(1);
    w.ts = c.take<TikState>(1);
    w.counters = c.take<unsigned>(k_max + 1);
    w.res2 = c.take<double>((long)(k_max + 1) * h * pb);
    w.fout = c.take<double>(h);
    w.cc = c.take<T>(h * k_max);
    w.zz = c.take<T>(h * (k_max + 1));
    w.tout = c.take<T>((long)TIK_P * h);
    w.lam = c.take<T>(TIK_P);
    w.tscr = c.take<T>((long)TIK_P * h * 4 * k_max);
    w.gv = p > 1 ? c.take<double>(h * pb * 3 * k_max) : nullptr;
    w.nA = rdft_parts(l, m);
    w.nB = rdft_parts(l, p);
    w.partsA = c.take<double>(w.nA);
    w.partsB = c.take<double>(w.nB);
    w.Ahat = c.take<V>(h * l * m);
    w.Bhat = c.take<V>(h * l * p);
    w.W = c.take<V>(h * pb * k_max * m);
    w.Q = c.take<V>(h * pb * (k_max + 1) * l);
    w.Xhat = c.take<V>(h * m * p);
    w.bytes = c.off;
    return w;
}

template <typename T>
static tp_status gk_check(int l, int m, int n, int p, const tp_tgkb_params* P) {
    if (!P || l < 1 || m < 1 || n < 1 || p < 1 || p > GKB_MAX_RHS) return TP_ERR_ARG;
    if (l > 1024 || m > 1024 || n > (sizeof(T) == 4 ? 1024 : 512)) return TP_ERR_ARG;
    const int mn = l < m ? l : m;
    if (P->k_max < 1 || P->k_max > mn || P->k_max > GKB_KMAX) return TP_ERR_ARG;
    if (!(P->tau > 0.0) || !(P->delta >= 0.0)) return TP_ERR_ARG;
    if (P->delta_p)
        for (int j = 0; j < p; ++j)
            if (!(P->delta_p[j] >= 0.0) || !isfinite(P->delta_p[j])) return TP_ERR_ARG;
    return TP_OK;
}

template <typename T>
size_t gk_ws_bytes(int l, int m, int n, int p, const tp_tgkb_params* P) {
    if (gk_check<T>(l, m, n, p, P) != TP_OK) return 0;
    return gk_carve<T>(nullptr, l, m, n, P->k_max, p).bytes;
}

#define TRY(x)                      \
    do {                            \
        tp_status _e = (x);         \
        if (_e != TP_OK) return _e; \
    } while (0)

// A-hat for a tGKB solve: the DFT of A into the workspace, or the caller's
// half spectrum (read only; ||A||^2 from it by Parseval for the non-finite
// input check).
template <typename T>
static tp_status gk_ahat(const T* A, const void* Ahat_in, int l, int m, int n, GkWs<T>& w, cudaStream_t st) {
    if (Ahat_in) {
        w.Ahat = (cplx<T>*)Ahat_in;
        return norm2_hat<T>(Ahat_in, n, l, m, w.partsA, st);
    }
    return rdft<T>(A, w.Ahat, n, l, m, m, (long)l * m, w.partsA, nullptr, st);
}

// One single-slice tGKB launch: column bs-strided B-hat of one lateral slice
// (Bhat_j, already offset) to its X-hat column (Xhat_j).
template <typename T>
static tp_status gk_single(const GkWs<T>& w, const cplx<T>* Bhat_j, cplx<T>* Xhat_j, int bs, int l, int m, int n,
                           int k_max, double td, tp_info* info, double* res_hist, int write_info, cudaStream_t st) {
    const int h = n / 2 + 1;
    if (cudaMemsetAsync(w.counters, 0, sizeof(unsigned) * (k_max + 1), st) != cudaSuccess) return TP_ERR_CUDA;
    const int L = l > m ? l : m;
    int dev = 0, nsm = 0, per_sm = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TP_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TP_ERR_CUDA;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) return TP_ERR_CUDA;
    // One CTA per Fourier slice, all resident (cooperative launch): 1024
    // threads when one CTA per SM suffices, else 512 (two per SM) or 256
    // (four per SM, up to n = 1214 on 152 SMs).  Vector loads need
    // 16-byte aligned rows.  Spare shared memory caches the first kc vectors
    // of both Krylov bases.
    const size_t vb = sizeof(cplx<T>);
    const int nt = (h <= nsm) ? 1024 : (h <= 2 * nsm ? 512 : 256);  // 1, 2 or 4 CTAs per SM
    const bool vec = ((size_t)m * vb) % 16 == 0 && (size_t)m * vb / 16 <= (size_t)nt;
    const size_t part_n = std::max<size_t>(4 * (size_t)L, 16 / vb * (size_t)nt);
    const size_t base_bytes = ((size_t)l + m + L + k_max + 1 + part_n) * vb;
    const size_t static_bytes = 24 * 1024;  // GkbShared and small arrays
    const size_t per_cta = (size_t)(228 * 1024) / (size_t)((h + nsm - 1) / nsm) - 2048;
    const size_t avail = per_cta > base_bytes + static_bytes ? per_cta - base_bytes - static_bytes : 0;
    // A shared-memory cache of the bases measured slower: it takes the L1
    // capacity that the streaming loads of A-hat need in flight.
    const int kc = 0 * (int)std::min<size_t>((size_t)k_max + 1, avail / (((size_t)l + m) * vb));
    const size_t smem = base_bytes + (size_t)kc * ((size_t)l + m) * vb;
    const void* kern;
    if (nt == 1024) kern = vec ? (const void*)k_gkb<T, true, 1024> : (const void*)k_gkb<T, false, 1024>;
    else if (nt == 512) kern = vec ? (const void*)k_gkb<T, true, 512> : (const void*)k_gkb<T, false, 512>;
    else kern = vec ? (const void*)k_gkb<T, true, 256> : (const void*)k_gkb<T, false, 256>;
    if (smem_optin(kern, smem) != TP_OK) return TP_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem) != cudaSuccess)
        return TP_ERR_CUDA;
    if (!coop || (long)per_sm * nsm < h) return TP_ERR_UNSUPPORTED;
    const cplx<T>* Ahat = w.Ahat;
    int l_ = l, m_ = m, n_ = n, h_ = h, k_ = k_max, wi = write_info, bs_ = bs;
    long long spin = wait_budget(4000000000LL);  // ~2 s at the GB300 SM clock
    int kc_ = kc, extra_ = wait_stall();
    void* args[] = {(void*)&Ahat, (void*)&Bhat_j, &l_, &m_, &n_, &h_, &k_, &td, (void*)&w.W, (void*)&w.Q,
                    (void*)&w.cc, (void*)&w.zz, (void*)&w.res2, (void*)&w.counters, (void*)&Xhat_j,
                    (void*)&w.st, (void*)&info, (void*)&res_hist, &spin, &wi, &kc_, &bs_, &extra_};
    prof_begin(TP_KC_GKB, st);
    if (cudaLaunchCooperativeKernel(kern, dim3(h), dim3(nt), args, smem, st) != cudaSuccess)
        return TP_ERR_CUDA;
    return launched(TP_KC_GKB, st);
}

template <typename T>
static tp_status gk_run(const T* A, const T* B, int l, int m, int n, const tp_tgkb_params* P, GkWs<T>& w,
                        tp_info* info, int write_info, cudaStream_t st, const void* Ahat_in = nullptr) {
    TRY(gk_ahat<T>(A, Ahat_in, l, m, n, w, st));
    TRY(rdft<T>(B, w.Bhat, n, l, 1, 1, l, w.partsB, nullptr, st));
    return gk_single<T>(w, w.Bhat, w.Xhat, 1, l, m, n, P->k_max, P->tau * P->delta, info, P->res_hist, write_info,
                        st);
}

// tGKB_p: p lateral slices, each with its own delta_j and k_j.  Groups of
// GKM_PB slices share the products with A in one batched launch; shapes that
// the batched kernel does not take run one single-slice launch per slice.
template <typename T>
static tp_status gk_run_p(const T* A, const T* B, int l, int m, int n, int p, const tp_tgkb_params* P, GkWs<T>& w,
                          tp_info* info, cudaStream_t st, const void* Ahat_in = nullptr) {
    const int h = n / 2 + 1, k_max = P->k_max;
    TRY(gk_ahat<T>(A, Ahat_in, l, m, n, w, st));
    TRY(rdft<T>(B, w.Bhat, n, l, p, p, (long)l * p, w.partsB, nullptr, st));
    auto td_of = [&](int j) { return P->tau * (P->delta_p ? P->delta_p[j] : P->delta); };
    int nt = 0;
    size_t smem = 0;
    const tp_status cfg = gkm_config<T>(l, m, n, k_max, &nt, &smem);
    if (cfg == TP_OK) {
        for (int j0 = 0; j0 < p; j0 += GKM_PB) {
            GkmArgs a;
            a.Ahat = w.Ahat;
            a.Bhat = w.Bhat;
            a.Wb = w.W;
            a.Qb = w.Q;
            a.Xhat = w.Xhat;
            a.gv = w.gv;
            a.res2 = w.res2;
            a.counters = w.counters;
            a.info = info;
            a.res_hist = P->res_hist;
            a.spin = wait_budget(4000000000LL);  // ~2 s at the GB300 SM clock
            a.extra = wait_stall();
            a.l = l;
            a.m = m;
            a.n = n;
            a.h = h;
            a.k_max = k_max;
            a.p = p;
            a.j0 = j0;
            a.pb = std::min(GKM_PB, p - j0);
            for (int j = 0; j < GKM_PB; ++j) {
                const double td = j < a.pb ? td_of(j0 + j) : 0.0;
                a.td[j] = td;
                a.td2n[j] = (double)n * td * td;
            }
            TRY(gkm_launch<T>(a, nt, smem, st));
        }
        return TP_OK;
    }
    if (cfg != TP_ERR_UNSUPPORTED) return cfg;
    const cplx<T>* Bh = w.Bhat;
    cplx<T>* Xh = w.Xhat;
    for (int j = 0; j < p; ++j)
        TRY(gk_single<T>(w, Bh + j, Xh + j, p, l, m, n, k_max, td_of(j), info + j,
                         P->res_hist ? P->res_hist + (long)j * (k_max + 1) : nullptr, 1, st));
    return TP_OK;
}

template <typename T>
tp_status gk_solve(const T* A, const T* B, int l, int m, int n, int p, const tp_tgkb_params* P, T* X,
                   tp_info* info, void* ws, size_t ws_bytes, cudaStream_t st, const void* Ahat) {
    TRY(gk_check<T>(l, m, n, p, P));
    if ((!A && !Ahat) || !B || !X || !info || ((size_t)Ahat & 15)) return TP_ERR_ARG;
    GkWs<T> w = gk_carve<T>(ws, l, m, n, P->k_max, p);
    if (!ws || ((size_t)ws & 255) || ws_bytes < w.bytes) return TP_ERR_WORKSPACE;
    if (p == 1) TRY(gk_run<T>(A, B, l, m, n, P, w, info, 1, st, Ahat));
    else TRY(gk_run_p<T>(A, B, l, m, n, p, P, w, info, st, Ahat));
    TRY(info_nonfinite(w.partsA, w.nA, w.partsB, w.nB, info, p, st));
    TRY(irdft<T>(w.Xhat, X, n, m, p, p, (long)m * p, nullptr, st));
    return TP_OK;
}

// ---- nested_tGKB_p host side ----------------------------------------------
template <typename T>
struct GknWs {
    unsigned* counters;
    double *res2, *phi, *rot, *td;
    double *partsA, *partsB;  // squared-norm partials of the DFTs (non-finite input check)
    int nA, nB;
    cplx<T> *Ahat, *Bhat, *W, *Q, *Xhat;
    size_t bytes;
};

template <typename T>
static GknWs<T> gkn_carve(void* base, int l, int m, int n, int k_max, int p) {
    typedef cplx<T> V;
    const long h = n / 2 + 1, ev = (long)k_max + p + 1;
    Carver c(base, 0);
    GknWs<T> w;
    w.counters = c.take<unsigned>(ev);
    w.res2 = c.take<double>(ev * h);
    w.phi = c.take<double>(h * k_max * 2);
    w.rot = c.take<double>(h * k_max * 3);
    w.td = c.take<double>(p);
    w.nA = rdft_parts(l, m);
    w.nB = rdft_parts(l, p);
    w.partsA = c.take<double>(w.nA);
    w.partsB = c.take<double>(w.nB);
    w.Ahat = c.take<V>(h * l * m);
    w.Bhat = c.take<V>(h * l * p);
    w.W = c.take<V>(h * (long)k_max * m);
    w.Q = c.take<V>(h * (long)(k_max + 1) * l);
    w.Xhat = c.take<V>(h * m * p);
    w.bytes = c.off;
    return w;
}

template <typename T>
size_t gkn_ws_bytes(int l, int m, int n, int p, const tp_tgkb_params* P) {
    if (gk_check<T>(l, m, n, p, P) != TP_OK) return 0;
    return gkn_carve<T>(nullptr, l, m, n, P->k_max, p).bytes;
}

struct TdChunk {
    double v[128];
};
__global__ void k_fill_td(double* dst, TdChunk c, int cnt) {
    if ((int)threadIdx.x < cnt) dst[threadIdx.x] = c.v[threadIdx.x];
}

template <typename T>
tp_status gkn_solve(const T* A, const T* B, int l, int m, int n, int p, const tp_tgkb_params* P, T* X,
                    tp_info* info, void* ws, size_t ws_bytes, cudaStream_t st) {
    TRY(gk_check<T>(l, m, n, p, P));
    if (!A || !B || !X || !info) return TP_ERR_ARG;
    const int h = n / 2 + 1, k_max = P->k_max, L = l > m ? l : m;
    GknWs<T> w = gkn_carve<T>(ws, l, m, n, k_max, p);
    if (!ws || ((size_t)ws & 255) || ws_bytes < w.bytes) return TP_ERR_WORKSPACE;
    int dev = 0, nsm = 0, per_sm = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TP_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TP_ERR_CUDA;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) return TP_ERR_CUDA;
    const size_t vb = sizeof(cplx<T>);
    const int nt = (h <= nsm) ? 1024 : (h <= 2 * nsm ? 512 : 256);  // 1, 2 or 4 CTAs per SM
    const bool vec = ((size_t)m * vb) % 16 == 0 && (size_t)m * vb / 16 <= (size_t)nt;
    const size_t part_n = std::max<size_t>(4 * (size_t)L, 16 / vb * (size_t)nt);
    const size_t smem = ((size_t)l + m + L + l + k_max + 1 + part_n) * vb;
    const void* kern;
    if (nt == 1024) kern = vec ? (const void*)k_gkb_nested<T, true, 1024> : (const void*)k_gkb_nested<T, false, 1024>;
    else if (nt == 512) kern = vec ? (const void*)k_gkb_nested<T, true, 512> : (const void*)k_gkb_nested<T, false, 512>;
    else kern = vec ? (const void*)k_gkb_nested<T, true, 256> : (const void*)k_gkb_nested<T, false, 256>;
    if (smem_optin(kern, smem) != TP_OK) return TP_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem) != cudaSuccess) return TP_ERR_CUDA;
    if (!coop || (long)per_sm * nsm < h) return TP_ERR_UNSUPPORTED;
    if (cudaMemsetAsync(w.counters, 0, sizeof(unsigned) * ((size_t)k_max + p + 1), st) != cudaSuccess)
        return TP_ERR_CUDA;
    for (int j0 = 0; j0 < p; j0 += 128) {  // eta delta_j, passed by value
        TdChunk c;
        const int cnt = std::min(128, p - j0);
        for (int j = 0; j < cnt; ++j) c.v[j] = P->tau * (P->delta_p ? P->delta_p[j0 + j] : P->delta);
        prof_begin(TP_KC_MISC, st);
        k_fill_td<<<1, 128, 0, st>>>(w.td + j0, c, cnt);
        TRY(launched(TP_KC_MISC, st));
    }
    TRY(rdft<T>(A, w.Ahat, n, l, m, m, (long)l * m, w.partsA, nullptr, st));
    TRY(rdft<T>(B, w.Bhat, n, l, p, p, (long)l * p, w.partsB, nullptr, st));
    GknArgs g;
    g.Ahat = w.Ahat;
    g.Bhat = w.Bhat;
    g.Wb = w.W;
    g.Qb = w.Q;
    g.Xhat = w.Xhat;
    g.phi = w.phi;
    g.rot = w.rot;
    g.res2 = w.res2;
    g.counters = w.counters;
    g.td = w.td;
    g.info = info;
    g.res_hist = P->res_hist;
    g.spin = wait_budget(4000000000LL);  // ~2 s at the GB300 SM clock
    g.extra = wait_stall();
    g.l = l;
    g.m = m;
    g.n = n;
    g.h = h;
    g.k_max = k_max;
    g.p = p;
    g.k_init = 2;  // Algorithm 6's k_init
    void* args[] = {(void*)&g};
    prof_begin(TP_KC_GKB, st);
    if (cudaLaunchCooperativeKernel(kern, dim3(h), dim3(nt), args, smem, st) != cudaSuccess) return TP_ERR_CUDA;
    TRY(launched(TP_KC_GKB, st));
    TRY(info_nonfinite(w.partsA, w.nA, w.partsB, w.nB, info, p, st));
    return irdft<T>(w.Xhat, X, n, m, p, p, (long)m * p, nullptr, st);
}

// ---- t-singular triplets from tGKB (Section 4.3, Eq. (solgkbb)) --------------
// k steps of Algorithm 4 from B; per Fourier slice the SVD of the (k+1) x k
// lower bidiagonal P_k (one-sided Jacobi on [P_k | 0], the rotations carried
// along an identity so that J comes out as well), then U = Q_{k+1} U_P and
// V = W_k V_P, and the inverse DFTs of U, the singular tubes and V.
template <typename T>
__global__ void k_bidiag(const T* cc, const T* zz, int k_max, const State* gst, cplx<T>* R, cplx<T>* D, int r,
                         State* st2) {
    const int s = blockIdx.x, ka = gst->k;  // the steps actually made (fewer after an exact breakdown)
    cplx<T>* Rs = R + (long)s * r * r;
    cplx<T>* Ds = D + (long)s * r * r;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int i = e / r, j = e - i * r;
        T v = 0;
        if (j < ka) {
            if (i == j) v = cc[(long)s * k_max + j];
            else if (i == j + 1) v = zz[(long)s * (k_max + 1) + j + 1];
        }
        Rs[e] = mk<T>(v, 0);
        Ds[e] = mk<T>(i == j ? (T)1 : (T)0, 0);
    }
    if (s == 0 && threadIdx.x == 0) {
        st2->r = r;
        st2->sweeps = 0;
    }
}

template <typename T>
__global__ void k_sigma_tubes(const T* sigma, int r, int k, cplx<T>* Sh) {
    const int s = blockIdx.x;
    for (int i = threadIdx.x; i < k; i += blockDim.x) Sh[(long)s * k + i] = mk<T>(sigma[(long)s * r + i], 0);
}

template <typename T>
struct TriWs {
    GkWs<T> g;
    State* st2;
    tp_info* info;
    T* sigma;
    cplx<T> *R, *D, *UR, *dprime, *Uh, *Vh, *Sh;
    size_t bytes;
};

template <typename T>
static TriWs<T> tri_carve(void* base, int l, int m, int n, int k) {
    typedef cplx<T> V;
    TriWs<T> w;
    w.g = gk_carve<T>(base, l, m, n, k, 1);
    const long h = n / 2 + 1, r = k + 1;
    Carver c(base ? (char*)base + w.g.bytes : nullptr, 0);
    w.st2 = c.take<State>(1);
    w.info = c.take<tp_info>(1);
    w.sigma = c.take<T>(h * r);
    w.R = c.take<V>(h * r * r);
    w.D = c.take<V>(h * r * r);
    w.UR = c.take<V>(h * r * r);
    w.dprime = c.take<V>(h * r * r);
    w.Uh = c.take<V>(h * l * k);
    w.Vh = c.take<V>(h * m * k);
    w.Sh = c.take<V>(h * k);
    w.bytes = w.g.bytes + c.off;
    return w;
}

template <typename T>
static tp_status tri_check(int l, int m, int n, int k) {
    tp_tgkb_params P = {0.0, 1.0, k, nullptr, nullptr};
    if (gk_check<T>(l, m, n, 1, &P) != TP_OK) return TP_ERR_ARG;
    // the Jacobi working set (r^2 + r^2 complex entries, r = k + 1) in shared memory
    if ((size_t)2 * (k + 1) * (k + 1) * sizeof(cplx<T>) + (size_t)(k + 1) * 12 > 227 * 1024) return TP_ERR_ARG;
    return TP_OK;
}

template <typename T>
size_t tri_ws_bytes(int l, int m, int n, int k) {
    if (tri_check<T>(l, m, n, k) != TP_OK) return 0;
    return tri_carve<T>(nullptr, l, m, n, k).bytes;
}

template <typename T>
tp_status tri_solve(const T* A, const T* B, int l, int m, int n, int k, T* U, T* S, T* V, void* ws, size_t ws_bytes,
                    cudaStream_t st) {
    TRY(tri_check<T>(l, m, n, k));
    if (!A || !B || !U || !S || !V) return TP_ERR_ARG;
    TriWs<T> w = tri_carve<T>(ws, l, m, n, k);
    if (!ws || ((size_t)ws & 255) || ws_bytes < w.bytes) return TP_ERR_WORKSPACE;
    const int h = n / 2 + 1, r = k + 1;
    // k steps of Algorithm 4 (delta = 0: no discrepancy stop before k)
    tp_tgkb_params P = {0.0, 1.0, k, nullptr, nullptr};
    TRY(gk_run<T>(A, B, l, m, n, &P, w.g, w.info, 0, st));
    prof_begin(TP_KC_MISC, st);
    k_bidiag<T><<<h, 256, 0, st>>>(w.g.cc, w.g.zz, k, w.g.st, w.R, w.D, r, w.st2);
    TRY(launched(TP_KC_MISC, st));
    TRY(jacobi_svd<T>(h, w.R, r, (long)r * r, w.st2, w.D, (long)r * r, r, w.sigma, r, w.UR, r, (long)r * r, w.dprime,
                      (long)r * r, r, &w.st2->sweeps, st));
    // U = Q_{k+1} U_P(:, 1:k);  V = W_k V_P(1:k, 1:k) with V_P = d'^H
    TRY(cgemm<T>(h, l, k, r, nullptr, nullptr, nullptr, 1, 0, w.g.Q, l, (long)(k + 1) * l, OP_T, w.UR, r,
                 (long)r * r, OP_N, 0, 0, w.Uh, k, (long)l * k, nullptr, st));
    TRY(cgemm<T>(h, m, k, k, nullptr, nullptr, nullptr, 1, 0, w.g.W, m, (long)k * m, OP_T, w.dprime, r,
                 (long)r * r, OP_C, 0, 0, w.Vh, k, (long)m * k, nullptr, st));
    prof_begin(TP_KC_MISC, st);
    k_sigma_tubes<T><<<h, 64, 0, st>>>(w.sigma, r, k, w.Sh);
    TRY(launched(TP_KC_MISC, st));
    TRY(irdft<T>(w.Uh, U, n, l, k, k, (long)l * k, nullptr, st));
    TRY(irdft<T>(w.Vh, V, n, m, k, k, (long)m * k, nullptr, st));
    return irdft<T>(w.Sh, S, n, 1, k, k, k, nullptr, st);
}

template size_t tri_ws_bytes<float>(int, int, int, int);
template size_t tri_ws_bytes<double>(int, int, int, int);
template tp_status tri_solve<float>(const float*, const float*, int, int, int, int, float*, float*, float*, void*,
                                    size_t, cudaStream_t);
template tp_status tri_solve<double>(const double*, const double*, int, int, int, int, double*, double*, double*,
                                     void*, size_t, cudaStream_t);

template <typename T>
size_t tik_ws_bytes(int l, int m, int n, int p, const tp_tik_params* P) {
    if (!P || p != 1) return 0;  // Tikhonov-tGKB: one lateral slice
    return gk_ws_bytes<T>(l, m, n, p, &P->gkb);
}

template <typename T>
tp_status tik_solve(const T* A, const T* B, int l, int m, int n, int p, const tp_tik_params* P, T* X,
                    tp_info* info, void* ws, size_t ws_bytes, cudaStream_t st, const void* Ahat) {
    if (!P || p != 1) return TP_ERR_ARG;
    TRY(gk_check<T>(l, m, n, p, &P->gkb));
    if (!(P->mu_lo > 0.0) || !(P->mu_hi > P->mu_lo)) return TP_ERR_ARG;
    if ((!A && !Ahat) || !B || !X || !info || ((size_t)Ahat & 15)) return TP_ERR_ARG;
    GkWs<T> w = gk_carve<T>(ws, l, m, n, P->gkb.k_max, 1);
    if (!ws || ((size_t)ws & 255) || ws_bytes < w.bytes) return TP_ERR_WORKSPACE;
    TRY(gk_run<T>(A, B, l, m, n, &P->gkb, w, info, 0, st, Ahat));
    const int h = n / 2 + 1, k_max = P->gkb.k_max;
    const double lo = log10(P->mu_lo), hi = log10(P->mu_hi);
    // the bracket is narrowed to log_tol, but no further than the spacing of
    // working-precision lam = mu^(-1/2) (float32: adjacent values differ by
    // 1e-7 in log10(mu), so narrower brackets hold one lam and change nothing)
    const double tol = std::max(P->log_tol > 0.0 ? P->log_tol : 1e-12, sizeof(T) == 4 ? 1e-7 : 0.0);
    const double td = P->gkb.tau * P->gkb.delta;
    const T thr = (T)((double)n * td * td);
    prof_begin(TP_KC_TIK, st);
    k_tik_init<T><<<1, TIK_P, 0, st>>>(w.ts, w.lam, lo, hi);
    TRY(launched(TP_KC_TIK, st));
    int rounds = 1;
    for (double width = hi - lo; width > tol && rounds < 40; width /= (TIK_P - 1)) ++rounds;
    // shared memory for the Givens data of up to tik_smem_k steps (k is known
    // on the device only; larger k use the global scratch)
    const size_t tsm = (size_t)3 * TIK_P * sizeof(T) * (size_t)std::min(k_max, tik_smem_k<T>());
    if (smem_optin((const void*)k_tik_round<T>, tsm) != TP_OK) return TP_ERR_CUDA;
    for (int it = 0; it < rounds; ++it) {
        prof_begin(TP_KC_TIK, st);
        k_tik_round<T><<<h, TIK_P, tsm, st>>>(w.cc, w.zz, k_max, w.st, w.ts, w.lam, h, n, w.tout, w.tscr, thr, tol);
        TRY(launched(TP_KC_TIK, st));
    }
    prof_begin(TP_KC_TIK, st);
    k_tik_final<T><<<h, 256, 0, st>>>(w.cc, w.zz, k_max, w.W, m, w.st, w.ts, n, w.fout, w.Xhat, w.tscr);
    TRY(launched(TP_KC_TIK, st));
    prof_begin(TP_KC_TIK, st);
    k_tik_info<<<1, 32, 0, st>>>(w.fout, h, n, w.st, w.ts, td, info);
    TRY(launched(TP_KC_TIK, st));
    TRY(info_nonfinite(w.partsA, w.nA, w.partsB, w.nB, info, 1, st));
    TRY(irdft<T>(w.Xhat, X, n, m, 1, 1, m, nullptr, st));
    return TP_OK;
}

// Tikhonov term of the tube-weight gradient, per slice s: with lam = 1/mu of
// the solve (mu = 10^t) and M = P^T P + lam I (P the (k+1) x k lower
// bidiagonal of the slice: c on the diagonal, z_1..z_k below it; M is
// tridiagonal with M_jj = c_j^2 + z_{j+1}^2 + lam, M_{j-1,j} = z_j c_j), the
// projected solution is y = M^{-1} P^T z_0 e_1 = M^{-1} (z_0 c_0) e_1 and
// dy/dlam = -M^{-1} y.  Then dX-hat/dlam = W_k dy/dlam and
//   add[s] = 2 lam Re<G-hat_s, W_k dy/dlam> = 2 lam sum_j dy_j Re(h_j),
// h_j = <w_j, G-hat_s>.  Warps form Re(h_j); one thread factors M = L D L^T
// (float64, positive pivots since lam > 0) and solves both systems.
// scr: per slice 3 k_max doubles.
template <typename T>
__global__ void __launch_bounds__(256) k_tik_rho(const T* cc, const T* zz, int k_max, const cplx<T>* Wb, int m,
                                                 const State* st, const TikState* ts, const cplx<T>* Gh,
                                                 double* scr, double* add) {
    __shared__ double hre[GKB_KMAX];
    const int s = blockIdx.x, k = st->k, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const cplx<T>* W = Wb + (long)s * k_max * m;
    const cplx<T>* g = Gh + (long)s * m;
    for (int j = warp; j < k; j += nw) {
        double a = 0.0;
        for (int e = lane; e < m; e += 32) {
            const cplx<T> w = W[(long)j * m + e], x = g[e];
            a += (double)(w.x * x.x + w.y * x.y);
        }
        a = warp_sum(a);
        if (lane == 0) hre[j] = a;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double lam = pow(10.0, -ts->t);
    const T* c = cc + (long)s * k_max;
    const T* z = zz + (long)s * (k_max + 1);
    double* dd = scr + (long)s * 3 * k_max;  // pivots of D
    double* ll = dd + k_max;                 // subdiagonal of L
    double* y = ll + k_max;
    for (int j = 0; j < k; ++j) {
        const double cj = (double)c[j], zj1 = (double)z[j + 1];
        const double mjj = cj * cj + zj1 * zj1 + lam;
        if (j == 0) {
            dd[0] = mjj;
        } else {
            const double off = (double)z[j] * cj;  // M_{j-1,j}
            ll[j] = off / dd[j - 1];
            dd[j] = mjj - ll[j] * off;
        }
    }
    // y = M^{-1} (z_0 c_0 e_1): forward with L, scale by D, back with L^T
    for (int j = 0; j < k; ++j) y[j] = j == 0 ? (double)z[0] * (double)c[0] : -ll[j] * y[j - 1];
    for (int j = 0; j < k; ++j) y[j] /= dd[j];
    for (int j = k - 2; j >= 0; --j) y[j] -= ll[j + 1] * y[j + 1];
    // dy = -M^{-1} y, accumulated into sum_j dy_j Re(h_j) on the way back
    double prev = 0.0;
    for (int j = 0; j < k; ++j) {
        const double u = -y[j] - (j > 0 ? ll[j] * prev : 0.0);
        prev = u;
        y[j] = u / dd[j];  // y now holds D^{-1} L^{-1} (-y)
    }
    double acc = 0.0, next = 0.0;
    for (int j = k - 1; j >= 0; --j) {
        const double dy = y[j] - (j + 1 < k ? ll[j + 1] * next : 0.0);
        next = dy;
        acc += dy * hre[j];
    }
    add[s] = 2.0 * lam * acc;
}

template <typename T>
static size_t tik_grad_carve(void* base, int m, int n, int k_max, cplx<T>** Gh, double2** gamma, double** add,
                             double** scr) {
    const size_t h = n / 2 + 1;
    Carver cv(base, 0);
    *Gh = cv.take<cplx<T>>(h * m);
    *gamma = cv.take<double2>(h);
    *add = cv.take<double>(h);
    *scr = cv.take<double>(h * 3 * (size_t)k_max);
    return cv.off;
}

template <typename T>
size_t tik_grad_ws_bytes(int l, int m, int n, const tp_tik_params* P) {
    if (!P || gk_check<T>(l, m, n, 1, &P->gkb) != TP_OK || n > GRAD_MAX_N) return 0;
    cplx<T>* Gh;
    double2* gamma;
    double *add, *scr;
    return tik_grad_carve<T>(nullptr, m, n, P->gkb.k_max, &Gh, &gamma, &add, &scr);
}

template <typename T>
tp_status tik_grad_c(const T* G, const double* c, int l, int m, int n, const tp_tik_params* P, const void* solve_ws,
                     size_t solve_ws_bytes, double* dc, void* ws, size_t ws_bytes, cudaStream_t st) {
    if (!P || !G || !c || !dc || n > GRAD_MAX_N) return TP_ERR_ARG;
    TRY(gk_check<T>(l, m, n, 1, &P->gkb));
    const int k_max = P->gkb.k_max, h = n / 2 + 1;
    GkWs<T> w = gk_carve<T>((void*)solve_ws, l, m, n, k_max, 1);
    if (!solve_ws || ((size_t)solve_ws & 255) || solve_ws_bytes < w.bytes) return TP_ERR_WORKSPACE;
    cplx<T>* Gh;
    double2* gamma;
    double *add, *scr;
    const size_t need = tik_grad_carve<T>(ws, m, n, k_max, &Gh, &gamma, &add, &scr);
    if (!ws || ((size_t)ws & 255) || ws_bytes < need) return TP_ERR_WORKSPACE;
    TRY(rdft<T>(G, Gh, n, m, 1, 1, m, nullptr, nullptr, st));
    prof_begin(TP_KC_MISC, st);
    k_tik_rho<T><<<h, 256, 0, st>>>(w.cc, w.zz, k_max, w.W, m, w.st, w.ts, Gh, scr, add);
    TRY(launched(TP_KC_MISC, st));
    TRY(sep_gamma<T>(w.Xhat, Gh, h, m, gamma, st));
    return grad_c(c, n, gamma, add, dc, st);
}

// ---------------------------------------------------------------------------
// dL/dB of the Tikhonov-tGKB solution at the k and mu of its solve: the
// reverse (adjoint) sweep through the k steps of Algorithm 4 per Fourier
// slice, with the two Gram-Schmidt passes and the Normalize steps, and
// through the projected Tikhonov solve y = M^{-1} P^T z_0 e_1 (M = P^T P +
// lam I, lam = 1/mu, P the (k+1) x k lower bidiagonal: c on the diagonal, z
// below).  The forward keeps the bases U (Q: u_0 .. u_k) and V (W: v_0 ..
// v_{k-1}); each step's intermediate vectors are recomputed from them (four
// products with A-hat per step).  Bars follow dL = Re<bar, d.> with dL/dx =
// G-hat_s; the sweep returns dL/db-hat_s, and dL/dB = irdft of those (the
// Parseval argument of the t-product's adjoint).  Float64 scalars; vectors
// and products in the working precision (the forward's); dot products summed
// in float64 across lanes.
// ---------------------------------------------------------------------------
constexpr int TIKADJ_THREADS = 512;

// out[i] = <Q_i, x> for i < cnt (Q_i = Q + i ld, length len): a warp per vector.
template <typename T>
__device__ void tadj_dots(const cplx<T>* Q, long ld, int cnt, const cplx<T>* x, int len, double2* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < cnt; i += nw) {
        const cplx<T>* q = Q + (long)i * ld;
        T ar = 0, ai = 0;
        for (int e = lane; e < len; e += 32) {
            const cplx<T> a = q[e], v = x[e];
            ar += a.x * v.x + a.y * v.y;
            ai += a.x * v.y - a.y * v.x;
        }
        const double r = warp_sum((double)ar), im = warp_sum((double)ai);
        if (lane == 0) out[i] = make_double2(r, im);
    }
    __syncthreads();
}

// Re<q, x> over len entries, every thread gets it (two barriers).
template <typename T>
__device__ double tadj_redot(const cplx<T>* q, const cplx<T>* x, int len, double* red) {
    T a = 0;
    for (int e = threadIdx.x; e < len; e += blockDim.x) a += q[e].x * x[e].x + q[e].y * x[e].y;
    return block_sum_t(a, red);
}

// Reverse of f = x - Q (Q^H x) over cnt basis vectors (c = Q^H x given):
// qf = Q^H fbar; Qbar_i -= fbar conj(c_i) + x conj(qf_i); xbar = fbar - Q qf
// (xbar may alias fbar).
template <typename T>
__device__ void tadj_unproj(const cplx<T>* Q, cplx<T>* Qbar, long ld, int cnt, int len, const double2* c,
                            double2* qf, const cplx<T>* fbar, const cplx<T>* x, cplx<T>* xbar) {
    tadj_dots<T>(Q, ld, cnt, fbar, len, qf);
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const cplx<T> fb = fbar[e], xv = x[e];
        T sr = 0, si = 0;  // the working precision (float64 arithmetic is 1/64 of the float32 rate)
        for (int i = 0; i < cnt; ++i) {
            const T cr = (T)c[i].x, ci = (T)c[i].y, qr = (T)qf[i].x, qi = (T)qf[i].y;
            cplx<T>* qb = Qbar + (long)i * ld + e;
            // fb conj(c_i) + x conj(qf_i)
            const T ur = fb.x * cr + fb.y * ci + xv.x * qr + xv.y * qi;
            const T ui = fb.y * cr - fb.x * ci + xv.y * qr - xv.x * qi;
            *qb = mk<T>(qb->x - ur, qb->y - ui);
            const cplx<T> q = Q[(long)i * ld + e];
            sr += q.x * qr - q.y * qi;
            si += q.x * qi + q.y * qr;
        }
        xbar[e] = mk<T>(fb.x - sr, fb.y - si);
    }
    __syncthreads();
}

// y[i] = sum_e a[i][e] v[e] - alpha u[i] (rows i < l of the l x m slice; a warp per row).
template <typename T>
__device__ void tadj_mv_n(const cplx<T>* a, int l, int m, const cplx<T>* v, double alpha, const cplx<T>* u,
                          cplx<T>* y) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < l; i += nw) {
        cplx<T> acc = mk<T>(0, 0);
        for (int e = lane; e < m; e += 32) cfma(acc, a[(long)i * m + e], v[e]);
        acc.x = warp_sum(acc.x);
        acc.y = warp_sum(acc.y);
        if (lane == 0) {
            if (u) acc = csub(acc, cscale(u[i], (T)alpha));
            y[i] = acc;
        }
    }
    __syncthreads();
}

// y[e] = sum_i conj(a[i][e]) t[i] - beta v[e] (columns e < m; a thread per column).
template <typename T>
__device__ void tadj_mv_c(const cplx<T>* a, int l, int m, const cplx<T>* t, double beta, const cplx<T>* v,
                          cplx<T>* y) {
    // columns e < m, the rows split into blockDim / m (at most 4) interleaved shares whose partial sums meet in
    // the shared array (fixed order); two accumulators per thread
    __shared__ cplx<T> part[3 * (TIKADJ_THREADS / 4)];  // (shares - 1) x span <= 3 x blockDim / 4
    int sh = (int)blockDim.x / m;
    sh = sh < 1 ? 1 : (sh > 4 ? 4 : sh);
    const int span = (int)blockDim.x / sh;  // threads per share
    const int share = (int)threadIdx.x / span, c0 = (int)threadIdx.x - share * span;
    for (int e0 = 0; e0 < m; e0 += span) {
        const int e = e0 + c0;
        cplx<T> acc0 = mk<T>(0, 0), acc1 = mk<T>(0, 0);
        if (share < sh && e < m) {
            int i = share;
            for (; i + sh < l; i += 2 * sh) {
                cfmac(acc0, a[(long)i * m + e], t[i]);
                cfmac(acc1, a[(long)(i + sh) * m + e], t[i + sh]);
            }
            if (i < l) cfmac(acc0, a[(long)i * m + e], t[i]);
        }
        const cplx<T> acc = cadd(acc0, acc1);
        if (share > 0 && share < sh && e < m) part[(share - 1) * span + c0] = acc;
        __syncthreads();
        if (share == 0 && e < m) {
            cplx<T> sum = acc;
            for (int q = 1; q < sh; ++q) sum = cadd(sum, part[(q - 1) * span + c0]);
            if (v) sum = csub(sum, cscale(v[e], (T)beta));
            y[e] = sum;
        }
        __syncthreads();
    }
}

// Reverse of (u, nrm) = (t / ||t||, ||t||): tbar = ubar / nrm + (nbar - Re<u, ubar> / nrm) u.
template <typename T>
__device__ void tadj_unnorm(const cplx<T>* ubar, double nbar, const cplx<T>* u, double nrm, int len, cplx<T>* tbar,
                            double* red) {
    const double ru = tadj_redot<T>(u, ubar, len, red);
    const T f = (T)(nbar - ru / nrm), in = (T)(1.0 / nrm);
    for (int e = threadIdx.x; e < len; e += blockDim.x)
        tbar[e] = mk<T>(ubar[e].x * in + f * u[e].x, ubar[e].y * in + f * u[e].y);
    __syncthreads();
}

template <typename T>
struct TadjArgs {
    const cplx<T>* Ahat;
    const cplx<T>* Ub;   // forward's Q: (h, k_max + 1, l)
    const cplx<T>* Vb;   // forward's W: (h, k_max, m)
    const T* cc;
    const T* zz;
    const State* st;
    const TikState* ts;
    const cplx<T>* Gh;   // (h, m)
    cplx<T>* Ubar;       // (h, k_max + 1, l)
    cplx<T>* Vbar;       // (h, k_max, m)
    cplx<T>* vec;        // (h, 3 l + 3 m): t0 t1 tb | w0 w1 wb
    double* sc;          // (h, 4 k_max + 2): y, s, albar, bebar
    cplx<T>* Yh;         // (h, l): dL/db-hat
    int l, m, k_max;
    int tik;             // 1: the Tikhonov solution (lam = 1/mu of the solve); 0: the tGKB solution (lam = 0)
};

template <typename T>
__global__ void __launch_bounds__(TIKADJ_THREADS) k_tikadj_rev(const TadjArgs<T> g) {
    typedef cplx<T> V;
    // first-pass coefficients (U^H t0, V^H w0), second-pass ones (U^H t1, V^H w1), and Q^H fbar
    __shared__ double2 cdot[GKB_KMAX + 1], c2[GKB_KMAX + 1], qf[GKB_KMAX + 1];
    __shared__ double red[33];
    const int s = blockIdx.x, tid = threadIdx.x, l = g.l, m = g.m, k_max = g.k_max;
    const int k = min(max(g.st->k, 0), k_max);  // a workspace that holds no solve cannot send the sweep out of bounds
    const V* a = g.Ahat + (long)s * l * m;
    const V* U = g.Ub + (long)s * (k_max + 1) * l;
    const V* Vv = g.Vb + (long)s * k_max * m;
    const T* c = g.cc + (long)s * k_max;
    const T* z = g.zz + (long)s * (k_max + 1);
    const V* G = g.Gh + (long)s * m;
    V* Ub = g.Ubar + (long)s * (k_max + 1) * l;
    V* Vb = g.Vbar + (long)s * k_max * m;
    V* t0 = g.vec + (long)s * (3 * l + 3 * m);
    V *t1 = t0 + l, *tb = t1 + l, *w0 = tb + l, *w1 = w0 + m, *wb = w1 + m;
    double* y = g.sc + (long)s * (4 * k_max + 2);
    double *sv = y + k_max, *albar = sv + k_max, *bebar = albar + k_max;
    const double lam = g.tik ? pow(10.0, -g.ts->t) : 0.0;

    // x = V y, y = M^{-1} P^T z_0 e_1:  ybar = Re(V^H G),  s = M^{-1} ybar,
    // Pbar = z_0 e_1 s^T - P (s y^T + y s^T),  Vbar = G y^T
    tadj_dots<T>(Vv, m, k, G, m, cdot);
    if (tid == 0) {
        double* dd = albar;  // scratch for the LDL^T pivots and multipliers (overwritten below)
        double* ll = bebar;
        for (int j = 0; j < k; ++j) {
            const double cj = (double)c[j], zj1 = (double)z[j + 1];
            const double mjj = cj * cj + zj1 * zj1 + lam;
            if (j == 0) {
                dd[0] = mjj;
            } else {
                const double off = (double)z[j] * cj;
                ll[j] = off / dd[j - 1];
                dd[j] = mjj - ll[j] * off;
            }
        }
        double py = 0.0, ps = 0.0;
        for (int j = 0; j < k; ++j) {
            const double fy = (j == 0 ? (double)z[0] * (double)c[0] : 0.0) - (j > 0 ? ll[j] * py : 0.0);
            const double fs = cdot[j].x - (j > 0 ? ll[j] * ps : 0.0);
            py = fy;
            ps = fs;
            y[j] = fy / dd[j];
            sv[j] = fs / dd[j];
        }
        for (int j = k - 2; j >= 0; --j) {
            y[j] -= ll[j + 1] * y[j + 1];
            sv[j] -= ll[j + 1] * sv[j + 1];
        }
        // the bars of the bidiagonal entries c_j = P[j][j] and z_{j+1} = P[j+1][j], and of z_0
        for (int j = 0; j < k; ++j) {
            double ab = -2.0 * (double)c[j] * sv[j] * y[j];
            if (j > 0) ab -= (double)z[j] * (sv[j - 1] * y[j] + y[j - 1] * sv[j]);
            if (j == 0) ab += (double)z[0] * sv[0];
            albar[j] = ab;
        }
        bebar[0] = sv[0] * (double)c[0];
        for (int j = 0; j < k; ++j) {
            double bb = -2.0 * (double)z[j + 1] * sv[j] * y[j];
            if (j + 1 < k) bb -= (double)c[j + 1] * (sv[j + 1] * y[j] + y[j + 1] * sv[j]);
            bebar[j + 1] = bb;
        }
    }
    __syncthreads();
    for (int e = tid; e < k * m; e += blockDim.x) {
        const int j = e / m, i = e - j * m;
        Vb[e] = cscale(G[i], (T)y[j]);
    }
    for (int e = tid; e < (k + 1) * l; e += blockDim.x) Ub[e] = mk<T>(0, 0);
    __syncthreads();

    for (int j = k - 1; j >= 0; --j) {
        const V* uj = U + (long)j * l;
        const V* vj = Vv + (long)j * m;
        const double aj = (double)c[j], bj1 = (double)z[j + 1];
        // forward of the step, recomputed: t0 = a v_j - c_j u_j, t1 = t0 - U (U^H t0) over u_0 .. u_j
        tadj_mv_n<T>(a, l, m, vj, aj, uj, t0);
        tadj_dots<T>(U, l, j + 1, t0, l, cdot);
        for (int e = tid; e < l; e += blockDim.x) {
            T sr = 0, si = 0;
            for (int i = 0; i <= j; ++i) {
                const V q = U[(long)i * l + e];
                const T cr = (T)cdot[i].x, ci = (T)cdot[i].y;
                sr += q.x * cr - q.y * ci;
                si += q.x * ci + q.y * cr;
            }
            t1[e] = mk<T>(t0[e].x - sr, t0[e].y - si);
        }
        __syncthreads();
        // u_{j+1} = t2 / z_{j+1};  t2 = t1 - U (U^H t1);  t1 = t0 - U (U^H t0)
        tadj_unnorm<T>(Ub + (long)(j + 1) * l, bebar[j + 1], U + (long)(j + 1) * l, bj1, l, tb, red);
        tadj_dots<T>(U, l, j + 1, t1, l, c2);
        tadj_unproj<T>(U, Ub, l, j + 1, l, c2, qf, tb, t1, tb);
        tadj_unproj<T>(U, Ub, l, j + 1, l, cdot, qf, tb, t0, tb);
        // t0 = a v_j - c_j u_j
        tadj_mv_c<T>(a, l, m, tb, 0.0, nullptr, w0);  // a^H t0bar into w0 (scratch)
        const double ru = tadj_redot<T>(uj, tb, l, red);
        for (int e = tid; e < m; e += blockDim.x) Vb[(long)j * m + e] = cadd(Vb[(long)j * m + e], w0[e]);
        for (int e = tid; e < l; e += blockDim.x) Ub[(long)j * l + e] = csub(Ub[(long)j * l + e], cscale(tb[e], (T)aj));
        if (tid == 0) albar[j] -= ru;
        __syncthreads();
        // forward, recomputed: w0 = a^H u_j - z_j v_{j-1}, w1 = w0 - V (V^H w0) over v_0 .. v_{j-1}
        tadj_mv_c<T>(a, l, m, uj, j > 0 ? (double)z[j] : 0.0, j > 0 ? Vv + (long)(j - 1) * m : nullptr, w0);
        tadj_dots<T>(Vv, m, j, w0, m, cdot);
        for (int e = tid; e < m; e += blockDim.x) {
            T sr = 0, si = 0;
            for (int i = 0; i < j; ++i) {
                const V q = Vv[(long)i * m + e];
                const T cr = (T)cdot[i].x, ci = (T)cdot[i].y;
                sr += q.x * cr - q.y * ci;
                si += q.x * ci + q.y * cr;
            }
            w1[e] = mk<T>(w0[e].x - sr, w0[e].y - si);
        }
        __syncthreads();
        // v_j = w2 / c_j;  w2 = w1 - V (V^H w1);  w1 = w0 - V (V^H w0)
        tadj_unnorm<T>(Vb + (long)j * m, albar[j], vj, aj, m, wb, red);
        tadj_dots<T>(Vv, m, j, w1, m, c2);
        tadj_unproj<T>(Vv, Vb, m, j, m, c2, qf, wb, w1, wb);
        tadj_unproj<T>(Vv, Vb, m, j, m, cdot, qf, wb, w0, wb);
        // w0 = a^H u_j - z_j v_{j-1}
        tadj_mv_n<T>(a, l, m, wb, 0.0, nullptr, t1);  // a w0bar into t1 (scratch)
        double rv = 0.0;
        if (j > 0) rv = tadj_redot<T>(Vv + (long)(j - 1) * m, wb, m, red);
        for (int e = tid; e < l; e += blockDim.x) Ub[(long)j * l + e] = cadd(Ub[(long)j * l + e], t1[e]);
        if (j > 0)
            for (int e = tid; e < m; e += blockDim.x)
                Vb[(long)(j - 1) * m + e] = csub(Vb[(long)(j - 1) * m + e], cscale(wb[e], (T)z[j]));
        if (tid == 0 && j > 0) bebar[j] -= rv;
        __syncthreads();
    }
    // u_0 = b / z_0
    tadj_unnorm<T>(Ub, bebar[0], U, (double)z[0], l, g.Yh + (long)s * l, red);
}

template <typename T>
static size_t tik_adj_carve(void* base, int l, int m, int n, int k_max, TadjArgs<T>* a) {
    const size_t h = n / 2 + 1;
    Carver cv(base, 0);
    a->Gh = cv.take<cplx<T>>(h * m);
    a->Ubar = cv.take<cplx<T>>(h * (k_max + 1) * (size_t)l);
    a->Vbar = cv.take<cplx<T>>(h * (size_t)k_max * m);
    a->vec = cv.take<cplx<T>>(h * (3 * (size_t)l + 3 * (size_t)m));
    a->Yh = cv.take<cplx<T>>(h * (size_t)l);
    a->sc = cv.take<double>(h * (4 * (size_t)k_max + 2));
    return cv.off;
}

template <typename T>
static size_t tadj_ws(int l, int m, int n, const tp_tgkb_params* P) {
    if (!P || gk_check<T>(l, m, n, 1, P) != TP_OK) return 0;
    TadjArgs<T> a;
    return tik_adj_carve<T>(nullptr, l, m, n, P->k_max, &a);
}

// The reverse sweep for the solution left in solve_ws by a single-slice tGKB
// (tik = 0) or Tikhonov-tGKB (tik = 1) solve with the same sizes and k_max.
template <typename T>
static tp_status tadj_run(const T* G, int l, int m, int n, const tp_tgkb_params* P, int tik, const void* solve_ws,
                          size_t solve_ws_bytes, const void* Ahat, T* dB, void* ws, size_t ws_bytes, cudaStream_t st) {
    if (!P || !G || !dB || ((size_t)Ahat & 15)) return TP_ERR_ARG;
    TRY(gk_check<T>(l, m, n, 1, P));
    const int k_max = P->k_max, h = n / 2 + 1;
    GkWs<T> w = gk_carve<T>((void*)solve_ws, l, m, n, k_max, 1);
    if (!solve_ws || ((size_t)solve_ws & 255) || solve_ws_bytes < w.bytes) return TP_ERR_WORKSPACE;
    TadjArgs<T> a;
    const size_t need = tik_adj_carve<T>(ws, l, m, n, k_max, &a);
    if (!ws || ((size_t)ws & 255) || ws_bytes < need) return TP_ERR_WORKSPACE;
    a.Ahat = Ahat ? (const cplx<T>*)Ahat : w.Ahat;  // the half spectrum the solve used
    a.Ub = w.Q;
    a.Vb = w.W;
    a.cc = w.cc;
    a.zz = w.zz;
    a.st = w.st;
    a.ts = w.ts;
    a.l = l;
    a.m = m;
    a.k_max = k_max;
    a.tik = tik;
    TRY(rdft<T>(G, (void*)a.Gh, n, m, 1, 1, m, nullptr, nullptr, st));
    prof_begin(TP_KC_MISC, st);
    k_tikadj_rev<T><<<h, TIKADJ_THREADS, 0, st>>>(a);
    TRY(launched(TP_KC_MISC, st));
    return irdft<T>(a.Yh, dB, n, l, 1, 1, l, nullptr, st);
}

template <typename T>
size_t tik_adj_ws_bytes(int l, int m, int n, const tp_tik_params* P) {
    return P ? tadj_ws<T>(l, m, n, &P->gkb) : 0;
}

template <typename T>
tp_status tik_adjoint(const T* G, int l, int m, int n, const tp_tik_params* P, const void* solve_ws,
                      size_t solve_ws_bytes, const void* Ahat, T* dB, void* ws, size_t ws_bytes, cudaStream_t st) {
    if (!P) return TP_ERR_ARG;
    return tadj_run<T>(G, l, m, n, &P->gkb, 1, solve_ws, solve_ws_bytes, Ahat, dB, ws, ws_bytes, st);
}

template <typename T>
size_t gk_adj_ws_bytes(int l, int m, int n, const tp_tgkb_params* P) {
    return tadj_ws<T>(l, m, n, P);
}

template <typename T>
tp_status gk_adjoint(const T* G, int l, int m, int n, const tp_tgkb_params* P, const void* solve_ws,
                     size_t solve_ws_bytes, const void* Ahat, T* dB, void* ws, size_t ws_bytes, cudaStream_t st) {
    return tadj_run<T>(G, l, m, n, P, 0, solve_ws, solve_ws_bytes, Ahat, dB, ws, ws_bytes, st);
}

template size_t gk_adj_ws_bytes<float>(int, int, int, const tp_tgkb_params*);
template size_t gk_adj_ws_bytes<double>(int, int, int, const tp_tgkb_params*);
template tp_status gk_adjoint<float>(const float*, int, int, int, const tp_tgkb_params*, const void*, size_t,
                                     const void*, float*, void*, size_t, cudaStream_t);
template tp_status gk_adjoint<double>(const double*, int, int, int, const tp_tgkb_params*, const void*, size_t,
                                      const void*, double*, void*, size_t, cudaStream_t);
template size_t tik_adj_ws_bytes<float>(int, int, int, const tp_tik_params*);
template size_t tik_adj_ws_bytes<double>(int, int, int, const tp_tik_params*);
template tp_status tik_adjoint<float>(const float*, int, int, int, const tp_tik_params*, const void*, size_t,
                                      const void*, float*, void*, size_t, cudaStream_t);
template tp_status tik_adjoint<double>(const double*, int, int, int, const tp_tik_params*, const void*, size_t,
                                       const void*, double*, void*, size_t, cudaStream_t);

template size_t tik_grad_ws_bytes<float>(int, int, int, const tp_tik_params*);
template size_t tik_grad_ws_bytes<double>(int, int, int, const tp_tik_params*);
template tp_status tik_grad_c<float>(const float*, const double*, int, int, int, const tp_tik_params*, const void*,
                                     size_t, double*, void*, size_t, cudaStream_t);
template tp_status tik_grad_c<double>(const double*, const double*, int, int, int, const tp_tik_params*, const void*,
                                      size_t, double*, void*, size_t, cudaStream_t);

template size_t gk_ws_bytes<float>(int, int, int, int, const tp_tgkb_params*);
template size_t gk_ws_bytes<double>(int, int, int, int, const tp_tgkb_params*);
template size_t gkn_ws_bytes<float>(int, int, int, int, const tp_tgkb_params*);
template size_t gkn_ws_bytes<double>(int, int, int, int, const tp_tgkb_params*);
template tp_status gkn_solve<float>(const float*, const float*, int, int, int, int, const tp_tgkb_params*, float*,
                                    tp_info*, void*, size_t, cudaStream_t);
template tp_status gkn_solve<double>(const double*, const double*, int, int, int, int, const tp_tgkb_params*,
                                     double*, tp_info*, void*, size_t, cudaStream_t);
template size_t tik_ws_bytes<float>(int, int, int, int, const tp_tik_params*);
template size_t tik_ws_bytes<double>(int, int, int, int, const tp_tik_params*);
template tp_status gk_solve<float>(const float*, const float*, int, int, int, int, const tp_tgkb_params*, float*,
                                   tp_info*, void*, size_t, cudaStream_t, const void*);
template tp_status gk_solve<double>(const double*, const double*, int, int, int, int, const tp_tgkb_params*,
                                    double*, tp_info*, void*, size_t, cudaStream_t, const void*);
template tp_status tik_solve<float>(const float*, const float*, int, int, int, int, const tp_tik_params*, float*,
                                    tp_info*, void*, size_t, cudaStream_t, const void*);
template tp_status tik_solve<double>(const double*, const double*, int, int, int, int, const tp_tik_params*,
                                     double*, tp_info*, void*, size_t, cudaStream_t, const void*);

}  // namespace tp
