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
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace tp {

constexpr int ORTH_THREADS = 256;
constexpr int JAC_THREADS = 512;
constexpr int MAX_BLOCK = 32;

// ---------------------------------------------------------------------------
// Block orthonormalisation (Algorithm 3, steps 5-9, in block form):
//   Y <- Y - Q (Q^H Y)   twice   (classical Gram-Schmidt against the basis)
//   then column by column: two CGS passes against the earlier block columns
//   and Normalize (a zero column stays zero).
// Y is L x b row-major per slice.  Optionally writes the result into the
// basis array (rows r_prev .. r_prev+b-1, vector-major), the R coefficients
// (rows 0..r_prev+b-1, columns r_prev.. of a row-major r_max x r_max matrix),
// and the float64 squared norm of the input block.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(ORTH_THREADS)
k_orth(cplx<T>* Y, long sY, int L, int b, const cplx<T>* Qb, long sQ, int r_prev, cplx<T>* Qout,
       cplx<T>* R, long ldr, long sR, int r_rows, double* normsq, const int* skip) {
    typedef cplx<T> V;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* Ys = (V*)smraw;                  // Ys[j*L + row]
    V* Cs = Ys + (size_t)b * L;         // r_prev x b, summed over both passes
    V* Cp = Cs + (size_t)r_prev * b;    // r_prev x b, this pass
    V* cb = Cp + (size_t)r_prev * b;    // MAX_BLOCK
    V* Rb = cb + MAX_BLOCK;             // b x b
    __shared__ double red[ORTH_THREADS / 32];
    __shared__ double bcast;
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    Y += (long)s * sY;

    double nn = 0.0;
    for (int e = tid; e < L * b; e += blockDim.x) {
        const int row = e / b, j = e - row * b;
        const V v = Y[e];
        Ys[(size_t)j * L + row] = v;
        nn += cabs2d(v);
    }
    for (int e = tid; e < b * b; e += blockDim.x) Rb[e] = mk<T>(0, 0);
    nn = block_sum(nn, red);
    if (normsq && tid == 0) normsq[s] = nn;

    if (r_prev > 0) {
        const V* Q = Qb + (long)s * sQ;
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = warp; i < r_prev; i += nw) {
                V acc[MAX_BLOCK];
#pragma unroll
                for (int j = 0; j < MAX_BLOCK; ++j) acc[j] = mk<T>(0, 0);
                for (int row = lane; row < L; row += 32) {
                    const V q = Q[(long)i * L + row];
#pragma unroll
                    for (int j = 0; j < MAX_BLOCK; ++j)
                        if (j < b) cfmac(acc[j], q, Ys[(size_t)j * L + row]);
                }
#pragma unroll
                for (int j = 0; j < MAX_BLOCK; ++j) {
                    if (j < b) {
                        acc[j].x = warp_sum(acc[j].x);
                        acc[j].y = warp_sum(acc[j].y);
                    }
                }
                if (lane == 0)
                    for (int j = 0; j < b; ++j) Cp[(size_t)i * b + j] = acc[j];
            }
            __syncthreads();
            for (int row = tid; row < L; row += blockDim.x) {
                V acc[MAX_BLOCK];
#pragma unroll
                for (int j = 0; j < MAX_BLOCK; ++j) acc[j] = mk<T>(0, 0);
                for (int i = 0; i < r_prev; ++i) {
                    const V q = Q[(long)i * L + row];
#pragma unroll
                    for (int j = 0; j < MAX_BLOCK; ++j)
                        if (j < b) cfma(acc[j], q, Cp[(size_t)i * b + j]);
                }
#pragma unroll
                for (int j = 0; j < MAX_BLOCK; ++j)
                    if (j < b) Ys[(size_t)j * L + row] = csub(Ys[(size_t)j * L + row], acc[j]);
            }
            for (int e = tid; e < r_prev * b; e += blockDim.x) Cs[e] = pass ? cadd(Cs[e], Cp[e]) : Cp[e];
            __syncthreads();
        }
    }

    for (int j = 0; j < b; ++j) {
        V* yj = Ys + (size_t)j * L;
        if (j > 0) {
            for (int pass = 0; pass < 2; ++pass) {
                for (int i = warp; i < j; i += nw) {
                    V acc = mk<T>(0, 0);
                    const V* yi = Ys + (size_t)i * L;
                    for (int row = lane; row < L; row += 32) cfmac(acc, yi[row], yj[row]);
                    acc.x = warp_sum(acc.x);
                    acc.y = warp_sum(acc.y);
                    if (lane == 0) cb[i] = acc;
                }
                __syncthreads();
                for (int row = tid; row < L; row += blockDim.x) {
                    V acc = mk<T>(0, 0);
                    for (int i = 0; i < j; ++i) cfma(acc, Ys[(size_t)i * L + row], cb[i]);
                    yj[row] = csub(yj[row], acc);
                }
                if (tid < j) Rb[tid * b + j] = cadd(Rb[tid * b + j], cb[tid]);
                __syncthreads();
            }
        }
        double p = 0.0;
        for (int row = tid; row < L; row += blockDim.x) p += cabs2d(yj[row]);
        p = block_sum(p, red);
        if (tid == 0) bcast = p;
        __syncthreads();
        const double nrm2 = bcast;
        const double inv = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
        for (int row = tid; row < L; row += blockDim.x) {
            const V v = yj[row];
            yj[row] = mk<T>((T)((double)v.x * inv), (T)((double)v.y * inv));
        }
        if (tid == 0) Rb[j * b + j] = mk<T>((T)sqrt(nrm2), 0);
        __syncthreads();
    }

    for (int e = tid; e < L * b; e += blockDim.x) {
        const int row = e / b, j = e - row * b;
        Y[e] = Ys[(size_t)j * L + row];
    }
    if (Qout) {
        V* Qo = Qout + (long)s * sQ + (long)r_prev * L;
        for (int e = tid; e < L * b; e += blockDim.x) Qo[e] = Ys[e];
    }
    if (R) {
        V* Rs = R + (long)s * sR;
        for (int e = tid; e < r_rows * b; e += blockDim.x) {
            const int i = e / b, j = e - i * b;
            V v = mk<T>(0, 0);  // rows below this block stay zero: R is block upper triangular
            if (i < r_prev) v = Cs[(size_t)i * b + j];
            else if (i < r_prev + b) v = Rb[(i - r_prev) * b + j];
            Rs[(long)i * ldr + r_prev + j] = v;
        }
    }
}

static size_t orth_smem(int L, int b, int r_prev, size_t c) {
    return ((size_t)b * L + 2 * (size_t)r_prev * b + MAX_BLOCK + (size_t)b * b) * c;
}

template <typename T>
static tp_status orth(int h, cplx<T>* Y, long sY, int L, int b, const cplx<T>* Qb, long sQ, int r_prev,
                      cplx<T>* Qout, cplx<T>* R, long ldr, long sR, int r_rows, double* normsq, const int* skip,
                      cudaStream_t st) {
    const size_t smem = orth_smem(L, b, r_prev, sizeof(cplx<T>));
    if (smem > 48 * 1024)
        if (cudaFuncSetAttribute(k_orth<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return TP_ERR_CUDA;
    prof_begin(TP_KC_ORTH, st);
    k_orth<T><<<h, ORTH_THREADS, smem, st>>>(Y, sY, L, b, Qb, sQ, r_prev, Qout, R, ldr, sR, r_rows, normsq, skip);
    return launched(TP_KC_ORTH, st);
}

// ---------------------------------------------------------------------------
// Scalars: ||A||^2 from the DFT partials, eps^2, and the eta update of
// Algorithm 3 (eta <- eta - ||Bt(block)||_F^2, Parseval-weighted over slices).
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
        st->eps2 = eps > 0.0 ? eps * eps : eps_rel * eps_rel * a2;
        st->done = (st->eta < st->eps2) ? 1 : 0;
        st->r = 0;
        st->k = 0;
        st->status = TP_OK;
        st->sweeps = 0;
        st->sigma_max = 0.0;
    }
}

__global__ void k_eta_update(State* st, const double* normsq, int h, int n, int r_new) {
    if (st->done) return;
    __shared__ double red[32];
    double a = 0.0;
    for (int s = threadIdx.x; s < h; s += blockDim.x) a += parseval_w(s, n) * normsq[s];
    a = block_sum(a, red);
    if (threadIdx.x == 0) {
        st->eta -= a / (double)n;
        st->r = r_new;
        if (st->eta < st->eps2) st->done = 1;
    }
}

// ---------------------------------------------------------------------------
// One-sided Jacobi SVD of R (r x r) per slice, rotations from the right
// (cyclic round-robin ordering, r/2 disjoint pairs per round, one warp per
// pair).  Tracks d' = J^H d.  Outputs, sorted by decreasing sigma:
// sigma (r), U_R (r x r row-major, columns normalised), d'.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(JAC_THREADS)
k_jacobi(const cplx<T>* __restrict__ R, long ldr, long sR, const State* st, const cplx<T>* __restrict__ d, long sd,
         T* sigma, long ssig, cplx<T>* UR, long ldu, long sU, cplx<T>* dprime, long sdp, int max_sweeps,
         int* sweeps_out) {
    typedef cplx<T> V;
    const int r = st->r;
    if (r <= 0) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* Rs = (V*)smraw;                       // column j at Rs[j*r]
    V* dp = Rs + (size_t)r * r;
    double* sg = (double*)(dp + r);
    int* perm = (int*)(sg + r);
    __shared__ int rot_count;
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    R += (long)s * sR;
    for (int e = tid; e < r * r; e += blockDim.x) {
        const int i = e / r, j = e - i * r;
        Rs[(size_t)j * r + i] = R[(long)i * ldr + j];
    }
    for (int i = tid; i < r; i += blockDim.x) dp[i] = d[(long)s * sd + i];
    __syncthreads();

    const int rr = r + (r & 1);
    const T tol = (T)(4.0 * sqrt((double)r) * Eps<T>::v);
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (tid == 0) rot_count = 0;
        __syncthreads();
        for (int t = 0; t < rr - 1; ++t) {
            for (int kp = warp; kp < rr / 2; kp += nw) {
                int p, q;
                if (kp == 0) {
                    p = 0;
                    q = 1 + t;
                } else {
                    p = 1 + (t + kp) % (rr - 1);
                    q = 1 + (t - kp + (rr - 1)) % (rr - 1);
                }
                if (p > q) { const int x = p; p = q; q = x; }
                if (q >= r) continue;
                V* cp = Rs + (size_t)p * r;
                V* cq = Rs + (size_t)q * r;
                T a = 0, bq = 0;
                V g = mk<T>(0, 0);
                for (int i = lane; i < r; i += 32) {
                    const V x = cp[i], y = cq[i];
                    a += x.x * x.x + x.y * x.y;
                    bq += y.x * y.x + y.y * y.y;
                    cfmac(g, x, y);
                }
                a = warp_sum(a);
                bq = warp_sum(bq);
                g.x = warp_sum(g.x);
                g.y = warp_sum(g.y);
                const T ag = sqrt(g.x * g.x + g.y * g.y);
                if (ag > (T)0 && ag > tol * sqrt(a) * sqrt(bq)) {
                    const T zeta = (bq - a) / ((T)2 * ag);
                    const T tt = (zeta >= (T)0 ? (T)1 : (T)-1) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
                    const T c = (T)1 / sqrt((T)1 + tt * tt), sn = c * tt;
                    const V e = mk<T>(g.x / ag, g.y / ag);
                    const V ec = cconj(e);
                    for (int i = lane; i < r; i += 32) {
                        const V x = cp[i];
                        const V ey = cmul(ec, cq[i]);
                        cp[i] = mk<T>(c * x.x - sn * ey.x, c * x.y - sn * ey.y);
                        cq[i] = mk<T>(sn * x.x + c * ey.x, sn * x.y + c * ey.y);
                    }
                    if (lane == 0) {
                        const V x = dp[p];
                        const V ey = cmul(e, dp[q]);
                        dp[p] = mk<T>(c * x.x - sn * ey.x, c * x.y - sn * ey.y);
                        dp[q] = mk<T>(sn * x.x + c * ey.x, sn * x.y + c * ey.y);
                        atomicAdd(&rot_count, 1);
                    }
                }
            }
            __syncthreads();
        }
        const int rc = rot_count;
        __syncthreads();
        if (rc == 0) break;
    }
    for (int j = warp; j < r; j += nw) {
        double a = 0.0;
        for (int i = lane; i < r; i += 32) a += cabs2d(Rs[(size_t)j * r + i]);
        a = warp_sum(a);
        if (lane == 0) sg[j] = sqrt(a);
    }
    __syncthreads();
    for (int j = tid; j < r; j += blockDim.x) {
        int rank = 0;
        const double v = sg[j];
        for (int i = 0; i < r; ++i) rank += (sg[i] > v) || (sg[i] == v && i < j);
        perm[rank] = j;
    }
    __syncthreads();
    for (int jr = tid; jr < r; jr += blockDim.x) {
        const int j = perm[jr];
        sigma[(long)s * ssig + jr] = (T)sg[j];
        dprime[(long)s * sdp + jr] = dp[j];
    }
    V* U = UR + (long)s * sU;
    for (int e = tid; e < r * r; e += blockDim.x) {
        const int i = e / r, jr = e - i * r;
        const int j = perm[jr];
        const double sv = sg[j];
        const V x = Rs[(size_t)j * r + i];
        U[(long)i * ldu + jr] = sv > 0.0 ? mk<T>((T)(x.x / sv), (T)(x.y / sv)) : mk<T>(0, 0);
    }
    if (tid == 0) atomicMax(sweeps_out, sweep + (sweep < max_sweeps ? 1 : 0));
}

static size_t jacobi_smem(int r, size_t c) {
    return (size_t)r * r * c + (size_t)r * c + (size_t)r * sizeof(double) + (size_t)r * sizeof(int);
}

// alpha_j = d'_j / sigma_j, dropping sigma_j <= dims * eps * sigma_max.
template <typename T>
__global__ void k_alpha(const T* sigma, long ssig, const cplx<T>* dprime, long sdp, cplx<T>* alpha, long sa,
                        const State* st, int h, int dims, int r_max) {
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
    for (int j = threadIdx.x; j < r_max; j += blockDim.x) {
        cplx<T> a = mk<T>(0, 0);
        if (j < r) {
            const double sv = (double)sigma[(long)s * ssig + j];
            if (sv > tol) {
                const cplx<T> v = dprime[(long)s * sdp + j];
                a = mk<T>((T)(v.x / sv), (T)(v.y / sv));
            }
        }
        alpha[(long)s * sa + j] = a;
    }
}

// Per slice: squared residual norms ||b - sum_{j<k} K_j alpha_j||^2 for all
// k = 0..r, where K = A V (stored vector-major, K_j contiguous).
template <typename T>
__global__ void __launch_bounds__(256)
k_dp_scan(const cplx<T>* __restrict__ KhT, long sK, const cplx<T>* __restrict__ alpha, long sa,
          const cplx<T>* __restrict__ bhat, long sb, const State* st, int l, double* out, long so) {
    typedef cplx<T> V;
    constexpr int RPT = 4;  // rows per thread (l <= 1024)
    extern __shared__ __align__(16) unsigned char smraw[];
    double* wsum = (double*)smraw;  // [8][r+1]
    const int r = st->r, s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = blockDim.x >> 5;
    KhT += (long)s * sK;
    V res[RPT];
    double part = 0.0;
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        const int i = tid + u * blockDim.x;
        res[u] = (i < l) ? bhat[(long)s * sb + i] : mk<T>(0, 0);
        part += cabs2d(res[u]);
    }
    part = warp_sum(part);
    if (lane == 0) wsum[warp * (r + 1)] = part;
    for (int j = 0; j < r; ++j) {
        const V a = alpha[(long)s * sa + j];
        part = 0.0;
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int i = tid + u * blockDim.x;
            if (i < l) {
                const V kv = KhT[(long)j * l + i];
                res[u] = csub(res[u], cmul(kv, a));
                part += cabs2d(res[u]);
            }
        }
        part = warp_sum(part);
        if (lane == 0) wsum[warp * (r + 1) + j + 1] = part;
    }
    __syncthreads();
    for (int j = tid; j <= r; j += blockDim.x) {
        double a = 0.0;
        for (int w = 0; w < nw; ++w) a += wsum[w * (r + 1) + j];
        out[(long)s * so + j] = a;
    }
}

// Global residuals (Parseval over slices), the discrepancy-principle choice
// of k in [max(1, r-p), r], and the info record.
__global__ void k_dp_reduce(const double* out, long so, int h, int n, State* st, int p_over, double tau_delta,
                            tp_info* info, double* res_hist, int r_max) {
    extern __shared__ double res[];
    const int r = st->r;
    for (int k = threadIdx.x; k <= r; k += blockDim.x) {
        double a = 0.0;
        for (int s = 0; s < h; ++s) a += parseval_w(s, n) * out[(long)s * so + k];
        res[k] = sqrt(fmax(a, 0.0) / (double)n);
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int k_init = max(1, r - p_over);
    int k = r, status = TP_ERR_NOT_CONVERGED;
    for (int j = k_init; j <= r; ++j)
        if (res[j] <= tau_delta) {
            k = j;
            status = TP_OK;
            break;
        }
    if (st->eta >= st->eps2) status = TP_ERR_NOT_CONVERGED;
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
    o.residual = res[k];
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
    cplx<T> *Ahat, *Bhat, *G, *Y, *Z, *Q, *BHb, *QG, *R, *d, *UR, *dprime, *alpha, *Vt, *KhT, *Xhat;
    T* sigma;
    size_t bytes;
};

template <typename T>
static RtWs<T> rt_carve(void* base, int l, int m, int n, int b, int r_max) {
    typedef cplx<T> V;
    const long h = n / 2 + 1;
    Carver c(base, 0);
    RtWs<T> w;
    w.st = c.take<State>(1);
    w.partsA = c.take<double>(rdft_parts(l, m));
    w.partsB = c.take<double>(rdft_parts(l, 1));
    w.normsq = c.take<double>(h);
    w.dpout = c.take<double>(h * (r_max + 1));
    w.Ahat = c.take<V>(h * l * m);
    w.Bhat = c.take<V>(h * l);
    w.G = c.take<V>(h * m * b);
    w.Y = c.take<V>(h * l * b);
    w.Z = c.take<V>(h * m * b);
    w.Q = c.take<V>(h * r_max * l);
    w.BHb = c.take<V>(h * m * b);
    w.QG = c.take<V>(h * r_max * m);
    w.R = c.take<V>(h * r_max * r_max);
    w.d = c.take<V>(h * r_max);
    w.UR = c.take<V>(h * r_max * r_max);
    w.dprime = c.take<V>(h * r_max);
    w.alpha = c.take<V>(h * r_max);
    w.Vt = c.take<V>(h * m * r_max);
    w.KhT = c.take<V>(h * r_max * l);
    w.Xhat = c.take<V>(h * m);
    w.sigma = c.take<T>(h * r_max);
    w.bytes = c.off;
    return w;
}

static int jac_rmax(size_t elem) {
    // largest r whose Jacobi working set fits in 227 KB of shared memory
    int r = 1;
    while (jacobi_smem(r + 1, 2 * elem) <= 227 * 1024) ++r;
    return r;
}

template <typename T>
static tp_status rt_check(int l, int m, int n, int p, const tp_rtsvd_params* P) {
    if (!P || l < 1 || m < 1 || n < 1 || p != 1) return TP_ERR_ARG;
    if (l > 1024 || m > 1024 || n > (sizeof(T) == 4 ? 1024 : 512)) return TP_ERR_ARG;
    if (P->block < 1 || P->block > MAX_BLOCK || P->r_max < 1 || P->r_max > (l < m ? l : m)) return TP_ERR_ARG;
    if (P->r_max > (sizeof(T) == 4 ? 160 : 112) || P->r_max > jac_rmax(sizeof(T))) return TP_ERR_ARG;
    if (!(P->tau > 0.0) || !(P->delta >= 0.0) || P->p_over < 0 || P->q_power < 0) return TP_ERR_ARG;
    if (!(P->eps > 0.0) && !(P->eps_rel > 0.0)) return TP_ERR_ARG;
    const int Lmax = l > m ? l : m;
    if (orth_smem(Lmax, P->block, P->r_max, 2 * sizeof(T)) > 227 * 1024) return TP_ERR_ARG;
    return TP_OK;
}

template <typename T>
size_t rt_ws_bytes(int l, int m, int n, int p, const tp_rtsvd_params* P) {
    if (rt_check<T>(l, m, n, p, P) != TP_OK) return 0;
    return rt_carve<T>(nullptr, l, m, n, P->block, P->r_max).bytes;
}

#define TRY(x)                              \
    do {                                    \
        tp_status _e = (x);                 \
        if (_e != TP_OK) return _e;         \
    } while (0)

template <typename T>
tp_status rt_solve(const T* A, const T* B, const T* Om, int l, int m, int n, int p, const tp_rtsvd_params* P, T* X,
                   tp_info* info, void* ws, size_t ws_bytes, cudaStream_t st) {
    TRY(rt_check<T>(l, m, n, p, P));
    if (!A || !B || !Om || !X || !info) return TP_ERR_ARG;
    const int b = P->block, r_max = P->r_max, h = n / 2 + 1;
    RtWs<T> w = rt_carve<T>(ws, l, m, n, b, r_max);
    if (!ws || ((size_t)ws & 255) || ws_bytes < w.bytes) return TP_ERR_WORKSPACE;
    const long lm = (long)l * m;
    const int* done = &w.st->done;

    TRY(rdft<T>(A, w.Ahat, n, l, m, m, lm, w.partsA, nullptr, st));
    TRY(rdft<T>(B, w.Bhat, n, l, 1, 1, l, w.partsB, nullptr, st));
    prof_begin(TP_KC_MISC, st);
    k_rt_init<<<1, 256, 0, st>>>(w.st, w.partsA, rdft_parts(l, m), w.partsB, rdft_parts(l, 1), P->eps, P->eps_rel, n);
    TRY(launched(TP_KC_MISC, st));

    const int nblk = (r_max + b - 1) / b;
    for (int blk = 0; blk < nblk; ++blk) {
        const int r0 = blk * b, bb = (b < r_max - r0) ? b : r_max - r0;
        // Gaussian block -> Fourier, sketch, power iterations, orthonormalise
        TRY(rdft<T>(Om + r0, w.G, n, m, bb, r_max, (long)m * r_max, nullptr, done, st));
        TRY(cgemm<T>(h, l, bb, m, 0, 0, 0, 1, 0, w.Ahat, m, lm, OP_N, w.G, bb, (long)m * bb, OP_N, 0, 0, w.Y, bb,
                     (long)l * bb, done, st));
        const bool last_y = (P->q_power == 0);
        TRY(orth<T>(h, w.Y, (long)l * bb, l, bb, w.Q, (long)r_max * l, r0, last_y ? w.Q : nullptr, nullptr, 0, 0, 0,
                    nullptr, done, st));
        for (int it = 0; it < P->q_power; ++it) {
            TRY(cgemm<T>(h, m, bb, l, 0, 0, 0, 1, 0, w.Ahat, m, lm, OP_C, w.Y, bb, (long)l * bb, OP_N, 0, 0, w.Z, bb,
                         (long)m * bb, done, st));
            TRY(orth<T>(h, w.Z, (long)m * bb, m, bb, nullptr, 0, 0, nullptr, nullptr, 0, 0, 0, nullptr, done, st));
            TRY(cgemm<T>(h, l, bb, m, 0, 0, 0, 1, 0, w.Ahat, m, lm, OP_N, w.Z, bb, (long)m * bb, OP_N, 0, 0, w.Y, bb,
                         (long)l * bb, done, st));
            const bool last = (it + 1 == P->q_power);
            TRY(orth<T>(h, w.Y, (long)l * bb, l, bb, w.Q, (long)r_max * l, r0, last ? w.Q : nullptr, nullptr, 0, 0,
                        0, nullptr, done, st));
        }
        // Bt(block)^H = A^H Y; its QR against the earlier columns extends QG and R
        TRY(cgemm<T>(h, m, bb, l, 0, 0, 0, 1, 0, w.Ahat, m, lm, OP_C, w.Y, bb, (long)l * bb, OP_N, 0, 0, w.BHb, bb,
                     (long)m * bb, done, st));
        TRY(orth<T>(h, w.BHb, (long)m * bb, m, bb, w.QG, (long)r_max * m, r0, w.QG, w.R, r_max,
                    (long)r_max * r_max, r_max, w.normsq, done, st));
        prof_begin(TP_KC_MISC, st);
        k_eta_update<<<1, 256, 0, st>>>(w.st, w.normsq, h, n, r0 + bb);
        TRY(launched(TP_KC_MISC, st));
    }
    const int* dr = &w.st->r;
    // d = Q^H b
    TRY(cgemm<T>(h, r_max, 1, l, dr, 0, 0, 1, 0, w.Q, l, (long)r_max * l, OP_R, w.Bhat, 1, l, OP_N, 0, 0, w.d, 1,
                 r_max, nullptr, st));
    {
        const size_t smem = jacobi_smem(r_max, sizeof(cplx<T>));
        if (smem > 48 * 1024)
            if (cudaFuncSetAttribute(k_jacobi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
                return TP_ERR_CUDA;
        prof_begin(TP_KC_SVD, st);
        k_jacobi<T><<<h, JAC_THREADS, smem, st>>>(w.R, r_max, (long)r_max * r_max, w.st, w.d, r_max, w.sigma, r_max,
                                                    w.UR, r_max, (long)r_max * r_max, w.dprime, r_max, 60,
                                                    &w.st->sweeps);
        TRY(launched(TP_KC_SVD, st));
    }
    prof_begin(TP_KC_MISC, st);
    k_alpha<T><<<h, 256, 0, st>>>(w.sigma, r_max, w.dprime, r_max, w.alpha, r_max, w.st, h, l > m ? l : m, r_max);
    TRY(launched(TP_KC_MISC, st));
    // V = QG^T-as-matrix * U_R ;  K^T = V^T A^T (vector-major K = A V)
    TRY(cgemm<T>(h, m, r_max, r_max, 0, dr, dr, 1, 0, w.QG, m, (long)r_max * m, OP_T, w.UR, r_max,
                 (long)r_max * r_max, OP_N, 0, 0, w.Vt, r_max, (long)m * r_max, nullptr, st));
    TRY(cgemm<T>(h, r_max, l, m, dr, 0, 0, 1, 0, w.Vt, r_max, (long)m * r_max, OP_T, w.Ahat, m, lm, OP_T, 0, 0,
                 w.KhT, l, (long)r_max * l, nullptr, st));
    {
        const size_t smem = (size_t)(256 / 32) * (r_max + 1) * sizeof(double);
        prof_begin(TP_KC_DP, st);
        k_dp_scan<T><<<h, 256, smem, st>>>(w.KhT, (long)r_max * l, w.alpha, r_max, w.Bhat, l, w.st, l, w.dpout,
                                           r_max + 1);
        TRY(launched(TP_KC_DP, st));
    }
    prof_begin(TP_KC_DP, st);
    k_dp_reduce<<<1, 256, (r_max + 1) * sizeof(double), st>>>(w.dpout, r_max + 1, h, n, w.st, P->p_over,
                                                              P->tau * P->delta, info, P->res_hist, r_max);
    TRY(launched(TP_KC_DP, st));
    TRY(cgemm<T>(h, m, 1, r_max, 0, 0, &w.st->k, 1, 0, w.Vt, r_max, (long)m * r_max, OP_N, w.alpha, 1, r_max, OP_N,
                 0, 0, w.Xhat, 1, m, nullptr, st));
    TRY(irdft<T>(w.Xhat, X, n, m, 1, 1, m, nullptr, st));
    return TP_OK;
}

template size_t rt_ws_bytes<float>(int, int, int, int, const tp_rtsvd_params*);
template size_t rt_ws_bytes<double>(int, int, int, int, const tp_rtsvd_params*);
template tp_status rt_solve<float>(const float*, const float*, const float*, int, int, int, int,
                                   const tp_rtsvd_params*, float*, tp_info*, void*, size_t, cudaStream_t);
template tp_status rt_solve<double>(const double*, const double*, const double*, int, int, int, int,
                                    const tp_rtsvd_params*, double*, tp_info*, void*, size_t, cudaStream_t);

}  // namespace tp
