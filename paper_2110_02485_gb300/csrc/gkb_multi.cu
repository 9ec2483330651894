// tGKB_p: the tGKB method for several lateral slices B_j of B (problem (I6)),
// each slice with its own noise bound delta_j and its own number of steps k_j
// (Sections 1 and 4.3: the method is applied to every slice separately).
//
// The slices are independent, but they share A: a launch carries a group of
// GKM_PB slices through Algorithm 4 in lockstep, so that both products of a
// step, A^H [q_1 .. q_PB] and A [w_1 .. w_PB], read each Fourier slice of A
// once for the whole group instead of once per lateral slice.  Everything
// else (reorthogonalisation, Normalize, the Givens QR of the projected
// problem, the discrepancy test) is per lateral slice, exactly as in the
// single-slice kernel: one CTA per Fourier slice, all resident (cooperative
// launch); after each step every CTA publishes one residual per lateral slice
// and waits (bounded) until all Fourier slices have done the step; every CTA
// then forms the same fixed-order sums and takes the same stop decisions.  A
// lateral slice that meets its bound stops (its step-i work is discarded, as
// in the single-slice kernel) while the others go on.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace tp {

// Partial reduce-scatter over lane bits 4, 3, 2 (eight lane groups of four):
// BB (>= 8) complex entries per lane; afterwards v[0 .. BB/8) of lane L hold
// the sums over the eight lanes L ^ (4 g) of entries (BB/8) (L >> 2) + t.
template <typename V, int BB>
__device__ __forceinline__ void reduce_scatter_hi3(V (&v)[BB]) {
    const int lane = threadIdx.x & 31;
    int cnt = BB;
#pragma unroll
    for (int o = 16; o >= 4; o >>= 1) {
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
    }
}

// u_j = A^H q_j - z_j w_j for the active lateral slices j of the group.  A
// warp takes four vector columns (4 VW columns) of A and eight row groups
// (lane = 4 g + c): every 16-byte load of A feeds all PB products; the row
// groups are combined by a partial reduce-scatter that leaves lane (g, c)
// with the VW results of lateral slice g.
template <typename T, int PB>
__device__ void mvh_multi(const cplx<T>* __restrict__ A, int l, int m, const cplx<T>* q, int lq, const cplx<T>* w,
                          int lw, const T* z, const int* act, cplx<T>* u, int lu) {
    typedef cplx<T> V;
    typedef typename Vec16<T>::type LV;
    constexpr int VW = Vec16<T>::VW, BB = PB * VW;
    static_assert(PB == 8, "lane group g writes lateral slice g");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c = lane & 3, g = lane >> 2;
    const int mv = m / VW, nch = (mv + 3) / 4;
    const LV* Av = (const LV*)A;
    for (int ch = warp; ch < nch; ch += nw) {
        const int cv = ch * 4 + c;
        const bool ok = cv < mv;
        V acc[BB];
#pragma unroll
        for (int e = 0; e < BB; ++e) acc[e] = mk<T>(0, 0);
        int i = g;
        for (; i + 8 < l; i += 16) {  // rows i and i + 8: two loads in flight
            LV a0, a1;
            if (ok) {
                a0 = __ldcg(Av + (long)i * mv + cv);
                a1 = __ldcg(Av + (long)(i + 8) * mv + cv);
            } else {
                a0 = a1 = LV{};
            }
            V e0[VW], e1[VW];
            unpack<T>(a0, e0);
            unpack<T>(a1, e1);
#pragma unroll
            for (int j = 0; j < PB; ++j) {
                const V q0 = q[j * lq + i], q1 = q[j * lq + i + 8];
#pragma unroll
                for (int v = 0; v < VW; ++v) {
                    cfmac(acc[j * VW + v], e0[v], q0);
                    cfmac(acc[j * VW + v], e1[v], q1);
                }
            }
        }
        if (i < l) {
            LV a0 = ok ? __ldcg(Av + (long)i * mv + cv) : LV{};
            V e0[VW];
            unpack<T>(a0, e0);
#pragma unroll
            for (int j = 0; j < PB; ++j) {
                const V q0 = q[j * lq + i];
#pragma unroll
                for (int v = 0; v < VW; ++v) cfmac(acc[j * VW + v], e0[v], q0);
            }
        }
        reduce_scatter_hi3<V, BB>(acc);
        if (ok && act[g]) {
            const T zg = z[g];
#pragma unroll
            for (int v = 0; v < VW; ++v) {
                const int col = cv * VW + v;
                u[g * lu + col] = csub(acc[v], cscale(w[g * lw + col], zg));
            }
        }
    }
    __syncthreads();
}

// u_j = A w_j - c_j q_j for the active lateral slices: a warp takes RB = 2
// consecutive rows, each lane a set of vector columns, and accumulates all
// 2 PB row sums; one reduce-scatter gives lane pair e the sum of entry e.
template <typename T, int PB>
__device__ void mvn_multi(const cplx<T>* __restrict__ A, int l, int m, const cplx<T>* w, int lw, const cplx<T>* q,
                          int lq, const T* cj, const int* act, cplx<T>* u, int lu) {
    typedef cplx<T> V;
    typedef typename Vec16<T>::type LV;
    constexpr int VW = Vec16<T>::VW, RB = 2, BB = RB * PB;
    static_assert(BB <= 32 && (BB & (BB - 1)) == 0, "reduce-scatter over one warp");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int mv = m / VW;
    const LV* Av = (const LV*)A;
    for (int i0 = warp * RB; i0 < l; i0 += nw * RB) {
        V acc[BB];
#pragma unroll
        for (int e = 0; e < BB; ++e) acc[e] = mk<T>(0, 0);
        const bool two = i0 + 1 < l;
        for (int cv = lane; cv < mv; cv += 32) {
            const LV a0 = __ldcg(Av + (long)i0 * mv + cv);
            const LV a1 = two ? __ldcg(Av + (long)(i0 + 1) * mv + cv) : LV{};
            V e0[VW], e1[VW];
            unpack<T>(a0, e0);
            unpack<T>(a1, e1);
#pragma unroll
            for (int j = 0; j < PB; ++j) {
                V wv[VW];
                unpack<T>(*(const LV*)(w + j * lw + cv * VW), wv);
#pragma unroll
                for (int v = 0; v < VW; ++v) {
                    cfma(acc[j], e0[v], wv[v]);
                    cfma(acc[PB + j], e1[v], wv[v]);
                }
            }
        }
        const V sum = warp_reduce_scatter<V, BB>(acc);
        const int e = lane / (32 / BB), r = e / PB, j = e - r * PB, i = i0 + r;
        if ((lane & (32 / BB - 1)) == 0 && i < l && act[j]) u[j * lu + i] = csub(sum, cscale(q[j * lq + i], cj[j]));
    }
    __syncthreads();
}

// Two classical Gram-Schmidt passes of u_j (length len) against the cnt
// basis vectors of lateral slice j (global, vector t at gb + j bsj + t len),
// for every active j.  cf: PB x cfs coefficient scratch.
template <typename T, int PB>
__device__ void reorth_multi(cplx<T>* u, int lu, int len, const cplx<T>* __restrict__ gb, long bsj, int cnt,
                             const int* act, cplx<T>* cf, int cfs) {
    typedef cplx<T> V;
    if (cnt <= 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5, NT = blockDim.x;
    for (int pass = 0; pass < 2; ++pass) {
        for (int it = warp; it < PB * cnt; it += nw) {
            const int j = it / cnt, t = it - j * cnt;
            if (!act[j]) continue;
            const V* bv = gb + j * bsj + (long)t * len;
            const V* uj = u + j * lu;
            V acc = mk<T>(0, 0);
#pragma unroll 4
            for (int e = lane; e < len; e += 32) cfmac(acc, __ldcg(bv + e), uj[e]);
            acc.x = warp_sum(acc.x);
            acc.y = warp_sum(acc.y);
            if (lane == 0) cf[j * cfs + t] = acc;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < PB * len; idx += NT) {
            const int j = idx / len, e = idx - j * len;
            if (!act[j]) continue;
            const V* bj = gb + j * bsj + e;
            const V* cfj = cf + j * cfs;
            V acc = mk<T>(0, 0);
#pragma unroll 4
            for (int t = 0; t < cnt; ++t) cfma(acc, __ldcg(bj + (long)t * len), cfj[t]);
            u[j * lu + e] = csub(u[j * lu + e], acc);
        }
        __syncthreads();
    }
}

// Normalize (per Fourier slice) of every active u_j: dst_j = u_j / ||u_j||
// in shared memory and at gdst + j gsj in global memory; nrm[j] = ||u_j||.  A
// zero vector gives zeros and norm 0.  Squares are summed in the working
// precision (one warp per lateral slice); the reciprocal falls back to
// float64 only when it is not finite for a positive sum.
template <typename T, int PB>
__device__ void normalize_multi(const cplx<T>* u, int lu, int len, cplx<T>* dst, int ld, cplx<T>* gdst, long gsj,
                                const int* act, T* nrm, T* inv, double* invd, int* mode) {
    typedef cplx<T> V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5, NT = blockDim.x;
    for (int j = warp; j < PB; j += nw) {
        if (!act[j]) continue;
        T p = 0;
        for (int e = lane; e < len; e += 32) p += cabs2(u[j * lu + e]);
        p = warp_sum(p);
        if (lane == 0) {
            const T iv = p > (T)0 ? (T)1 / sqrt(p) : (T)0;
            nrm[j] = sqrt(p);
            inv[j] = iv;
            mode[j] = (p > (T)0 && !isfinite(iv)) ? 1 : 0;
            if (mode[j]) invd[j] = 1.0 / sqrt((double)p);
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < PB * len; idx += NT) {
        const int j = idx / len, e = idx - j * len;
        if (!act[j]) continue;
        const V x = u[j * lu + e];
        V y;
        if (mode[j] == 0) {
            y = cscale(x, inv[j]);
        } else {
            const double iv = invd[j];
            y = mk<T>((T)((double)x.x * iv), (T)((double)x.y * iv));
        }
        dst[j * ld + e] = y;
        gdst[j * gsj + e] = y;
    }
    __syncthreads();
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, 1) k_gkb_multi(const GkmArgs a) {
    typedef cplx<T> V;
    constexpr int PB = GKM_PB, VW = Vec16<T>::VW;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int l = a.l, m = a.m, n = a.n, h = a.h, k_max = a.k_max, p = a.p, j0 = a.j0, pb = a.pb;
    const int L = l > m ? l : m;
    const int lq = (l + VW - 1) / VW * VW, lw = (m + VW - 1) / VW * VW, lu = (L + VW - 1) / VW * VW;
    const int cfs = k_max + 1;
    V* q = (V*)smraw;       // PB x lq: current q_j
    V* w = q + PB * lq;     // PB x lw: current w_j
    V* u = w + PB * lw;     // PB x lu: work vectors
    V* cf = u + PB * lu;    // PB x cfs: Gram-Schmidt coefficients, then y_j
    __shared__ T nrm[PB], inv[PB], cj[PB], zj[PB], zprev[PB];
    __shared__ double invd[PB], rcur[PB], rprev[PB];
    __shared__ int mode[PB], act[PB], kj[PB], done[PB];
    __shared__ int flag_timeout;
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const V* A = (const V*)a.Ahat + (long)s * l * m;
    const V* Bhat = (const V*)a.Bhat;
    V* Xhat = (V*)a.Xhat;
    V* Wg = (V*)a.Wb + (long)s * PB * k_max * m;          // lateral slice j: Wg + j k_max m
    V* Qg = (V*)a.Qb + (long)s * PB * (k_max + 1) * l;    // lateral slice j: Qg + j (k_max+1) l
    double* gv = a.gv + (long)s * PB * 3 * k_max;     // lateral slice j: rho, theta, phi
    const double ws = parseval_w(s, n);

    if (tid < PB) {
        act[tid] = tid < pb ? 1 : 0;
        kj[tid] = k_max;
        done[tid] = 0;
        rcur[tid] = rprev[tid] = -1.0;
        mode[tid] = 0;
    }
    if (tid == 0) flag_timeout = 0;
    for (int idx = tid; idx < PB * lu; idx += NT) {
        const int j = idx / lu, i = idx - j * lu;
        u[idx] = (j < pb && i < l) ? Bhat[((long)s * l + i) * p + j0 + j] : mk<T>(0, 0);
    }
    for (int idx = tid; idx < PB * lq; idx += NT) q[idx] = mk<T>(0, 0);
    for (int idx = tid; idx < PB * lw; idx += NT) w[idx] = mk<T>(0, 0);
    __syncthreads();
    normalize_multi<T, PB>(u, lu, l, q, lq, Qg, (long)(k_max + 1) * l, act, nrm, inv, invd, mode);
    // Givens state of lateral slice tid (threads 0..PB-1): phibar, previous
    // rotation, orphan residual
    // (rotations in the working precision, as in the single-slice kernel)
    T phibar = 0, cs_prev = 1, sn_prev = 0, orphan = 0;
    if (tid < PB) {
        phibar = act[tid] ? nrm[tid] : (T)0;
        zprev[tid] = act[tid] ? nrm[tid] : (T)0;
    }
    __syncthreads();

    for (int i = 1; i <= k_max + 1; ++i) {
        const bool step = i <= k_max;
        // W_i = A^T * Q_i - W_{i-1} * z_i for every lateral slice still going
        if (step) mvh_multi<T, PB>(A, l, m, q, lq, w, lw, zprev, act, u, lu);
        if (i >= 2) {
            if (tid == 0) {
                const long long t0 = clock64();
                while (ld_acquire(&a.counters[i - 1]) < (unsigned)(h + a.extra)) {
                    if (clock64() - t0 > a.spin) {
                        flag_timeout = 1;
                        break;
                    }
                }
            }
            __syncthreads();
            // residual of step i-1 per lateral slice: the same fixed-order sum
            // over Fourier slices in every CTA
            if (!flag_timeout) {
                for (int j = warp; j < PB; j += NT / 32) {
                    if (!act[j]) continue;
                    double tot = 0.0;
                    for (int s2 = lane; s2 < h; s2 += 32) tot += __ldcg(&a.res2[((long)(i - 1) * PB + j) * h + s2]);
                    tot = warp_sum(tot);
                    if (lane == 0) {
                        rprev[j] = rcur[j];
                        rcur[j] = tot;
                        if (s == 0 && a.res_hist) a.res_hist[(long)(j0 + j) * (k_max + 1) + i - 1] = sqrt(tot / n);
                        if (tot <= a.td2n[j]) {
                            act[j] = 0;
                            kj[j] = i - 1;
                            done[j] = 1;
                        }
                    }
                }
            }
            __syncthreads();
            if (flag_timeout) {
                if (tid < PB && act[tid]) {
                    kj[tid] = i - 1;
                    act[tid] = 0;
                }
                break;
            }
            if (!__syncthreads_or(tid < PB && act[tid])) break;
        }
        if (!step) break;
        // reorthogonalise; Normalize -> c_i, w = W_i
        reorth_multi<T, PB>(u, lu, m, Wg, (long)k_max * m, i - 1, act, cf, cfs);
        normalize_multi<T, PB>(u, lu, m, w, lw, Wg + (long)(i - 1) * m, (long)k_max * m, act, cj, inv, invd, mode);
        // Q_{i+1} = A * W_i - Q_i * c_i; reorthogonalise; Normalize -> z_{i+1}
        mvn_multi<T, PB>(A, l, m, w, lw, q, lq, cj, act, u, lu);
        reorth_multi<T, PB>(u, lu, l, Qg, (long)(k_max + 1) * l, i, act, cf, cfs);
        normalize_multi<T, PB>(u, lu, l, q, lq, Qg + (long)i * l, (long)(k_max + 1) * l, act, zj, inv, invd, mode);
        if (tid < PB && act[tid]) {
            // Givens QR of lateral slice tid's lower-bidiagonal slice: column i
            // has c_i on the diagonal and z_{i+1} below it
            double* gj = gv + (long)tid * 3 * k_max;
            const T cid = cj[tid], zid = zj[tid];
            const T rhobar = (i == 1) ? cid : cs_prev * cid;
            gj[k_max + i - 1] = (i == 1) ? 0.0 : (double)(sn_prev * cid);  // theta: R(i-1, i)
            const T rho = sqrt(fma(rhobar, rhobar, zid * zid));
            T c = 1, sn = 0;
            if (rho > (T)0) {
                const T irho = (T)1 / rho;
                c = rhobar * irho;
                sn = zid * irho;
                gj[2 * k_max + i - 1] = (double)(c * phibar);
                phibar = -sn * phibar;
            } else {  // zero column: its right-hand side entry stays unmatched
                gj[2 * k_max + i - 1] = 0.0;
                orphan += phibar * phibar;
                phibar = 0;
            }
            gj[i - 1] = rho;
            cs_prev = c;
            sn_prev = sn;
            a.res2[((long)i * PB + tid) * h + s] = ws * (double)(orphan + phibar * phibar);
            zprev[tid] = zj[tid];
            __threadfence();
        }
        __syncthreads();
        // step i done here (release after every lateral slice's residual)
        if (tid == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&a.counters[i]) : "memory");
    }
    __syncthreads();
    // back substitution R y = phi per lateral slice (float64), y kept in the
    // working precision for X-hat = W y
    T* yt = (T*)cf;
    if (tid < pb) {
        const double* gj = gv + (long)tid * 3 * k_max;
        const int k = kj[tid];
        double ynext = 0.0;
        for (int t = k - 1; t >= 0; --t) {
            double v = gj[2 * k_max + t];
            if (t + 1 < k) v -= gj[k_max + t + 1] * ynext;
            const double y = gj[t] > 0.0 ? v / gj[t] : 0.0;
            yt[tid * cfs + t] = (T)y;
            ynext = y;
        }
    }
    __syncthreads();
    for (int idx = tid; idx < pb * m; idx += NT) {
        const int j = idx / m, e = idx - j * m;
        const V* Wj = Wg + (long)j * k_max * m + e;
        const T* yj = yt + j * cfs;
        V x = mk<T>(0, 0);
        for (int t = 0; t < kj[j]; ++t) {
            const V v = Wj[(long)t * m];
            x.x = fma(v.x, yj[t], x.x);
            x.y = fma(v.y, yj[t], x.y);
        }
        Xhat[((long)s * m + e) * p + j0 + j] = x;
    }
    if (s == 0 && tid < pb) {
        const int k = kj[tid];
        const double td = a.td[tid];
        const int status = flag_timeout ? TP_ERR_TIMEOUT : (done[tid] ? TP_OK : TP_ERR_NOT_CONVERGED);
        const double res_k = flag_timeout ? -1.0 : sqrt(rcur[tid] / n);
        double margin = fabs(res_k - td) / td;
        if (k >= 2 && !flag_timeout) margin = fmin(margin, fabs(sqrt(rprev[tid] / n) - td) / td);
        if (a.res_hist) {
            double* rh = a.res_hist + (long)(j0 + tid) * (k_max + 1);
            rh[0] = -1.0;
            for (int t = k + 1; t <= k_max; ++t) rh[t] = -1.0;
            if (flag_timeout)
                for (int t = 1; t <= k; ++t) rh[t] = -1.0;
        }
        tp_info o;
        o.status = status;
        o.k = k;
        o.r = k;
        o.sweeps = 0;
        o.residual = res_k;
        o.tau_delta = td;
        o.eta = 0.0;
        o.mu = 0.0;
        o.margin = margin;
        o.norm_a2 = 0.0;
        a.info[j0 + tid] = o;
    }
}

// 1024 threads only for float data (the float64 accumulators need the
// registers of a 512-thread CTA)
template <typename T> static const void* gkm_kernel(int nt);
template <> const void* gkm_kernel<float>(int nt) {
    return nt == 1024 ? (const void*)k_gkb_multi<float, 1024> : (const void*)k_gkb_multi<float, 512>;
}
template <> const void* gkm_kernel<double>(int) { return (const void*)k_gkb_multi<double, 512>; }

static size_t gkm_smem(int l, int m, int k_max, size_t vb, int vw) {
    const int L = l > m ? l : m;
    const size_t lq = (l + vw - 1) / vw * vw, lw = (m + vw - 1) / vw * vw, lu = (L + vw - 1) / vw * vw;
    return (size_t)GKM_PB * (lq + lw + lu + (size_t)k_max + 1) * vb;
}

template <typename T>
tp_status gkm_config(int l, int m, int n, int k_max, int* nt_out, size_t* smem_out) {
    const size_t vb = sizeof(cplx<T>);
    const int vw = Vec16<T>::VW;
    // 16-byte loads of A need 16-byte rows
    if (((size_t)m * vb) % 16 != 0) return TP_ERR_UNSUPPORTED;
    const int h = n / 2 + 1;
    int dev = 0, nsm = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TP_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TP_ERR_CUDA;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) return TP_ERR_CUDA;
    if (!coop) return TP_ERR_UNSUPPORTED;
    const size_t smem = gkm_smem(l, m, k_max, vb, vw);
    if (smem > 200 * 1024) return TP_ERR_UNSUPPORTED;
    // float data: 1024 threads when one CTA per SM holds every Fourier slice
    for (int nt : {1024, 512}) {
        if (nt == 1024 && (sizeof(T) != 4 || h > nsm)) continue;
        const void* kern = gkm_kernel<T>(nt);
        if (smem_optin(kern, smem) != TP_OK) return TP_ERR_CUDA;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem) != cudaSuccess)
            return TP_ERR_CUDA;
        if ((long)per_sm * nsm >= h) {
            *nt_out = nt;
            *smem_out = smem;
            return TP_OK;
        }
    }
    return TP_ERR_UNSUPPORTED;
}

template <typename T>
tp_status gkm_launch(const GkmArgs& a, int nt, size_t smem, cudaStream_t st) {
    if (cudaMemsetAsync(a.counters, 0, sizeof(unsigned) * (a.k_max + 1), st) != cudaSuccess) return TP_ERR_CUDA;
    GkmArgs args = a;
    void* kargs[] = {(void*)&args};
    prof_begin(TP_KC_GKB, st);
    if (cudaLaunchCooperativeKernel(gkm_kernel<T>(nt), dim3(a.h), dim3(nt), kargs, smem, st) != cudaSuccess)
        return TP_ERR_CUDA;
    return launched(TP_KC_GKB, st);
}

template tp_status gkm_config<float>(int, int, int, int, int*, size_t*);
template tp_status gkm_config<double>(int, int, int, int, int*, size_t*);
template tp_status gkm_launch<float>(const GkmArgs&, int, size_t, cudaStream_t);
template tp_status gkm_launch<double>(const GkmArgs&, int, size_t, cudaStream_t);

}  // namespace tp
