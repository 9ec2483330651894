#include <atomic>
// extern "C" entry points of libtprod (declared in include/tprod.h).
#include <stdint.h>

#include "common.cuh"
#include "internal.h"

#include <mutex>
#include <unordered_map>
#include <vector>

namespace tp {

std::atomic<long long> g_wait_budget{0};
std::atomic<int> g_wait_stall{0};

long long wait_budget(long long dflt) {
    const long long v = g_wait_budget.load();
    return v > 0 ? v : dflt;
}

int wait_stall() { return g_wait_stall.load(); }

__global__ void k_info_nonfinite(const double* pa, int na, const double* pb, int nb, tp_info* info, int cnt) {
    __shared__ double red[33];
    double a = 0.0;
    for (int i = threadIdx.x; i < na; i += blockDim.x) a += pa[i];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) a += pb[i];
    a = block_sum_t(a, red);
    if (isfinite(a)) return;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        info[j].status = TP_ERR_NONFINITE;
        info[j].residual = __longlong_as_double(0x7ff8000000000000LL);  // NaN
    }
}

tp_status info_nonfinite(const double* partsA, int nA, const double* partsB, int nB, tp_info* info, int cnt,
                         cudaStream_t st) {
    prof_begin(TP_KC_MISC, st);
    k_info_nonfinite<<<1, 256, 0, st>>>(partsA, nA, partsB, nB, info, cnt);
    return launched(TP_KC_MISC, st);
}


int g_launches = 0;

// ---- optional per-class device timing -------------------------------------
namespace {
struct Rec {
    int cls;
    cudaEvent_t a, b;
};
int g_mask = 0;
std::vector<cudaEvent_t> g_pool;   // free events
std::vector<Rec> g_recs;           // recorded launches
int g_open_cls = -1;
cudaEvent_t g_open = nullptr;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

// Records e on st; inside a stream capture the record becomes a node of the
// graph (an external event record), so that every replay records it again.
static void record(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
}

void prof_begin(int cls, cudaStream_t st) {
    if (!(g_mask >> cls & 1)) return;
    g_open = take_event();
    g_open_cls = g_open ? cls : -1;
    if (g_open) record(g_open, st);
}

void prof_end(int cls, cudaStream_t st) {
    if (g_open_cls != cls || !g_open) return;
    cudaEvent_t e = take_event();
    if (e) {
        record(e, st);
        g_recs.push_back({cls, g_open, e});
    } else {
        g_pool.push_back(g_open);
    }
    g_open = nullptr;
    g_open_cls = -1;
}

tp_status smem_optin(const void* kern, size_t bytes) {
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> done;
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find(kern);
    if (it != done.end() && it->second >= bytes) return TP_OK;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return TP_ERR_CUDA;
    done[kern] = bytes;
    return TP_OK;
}

template <typename T> size_t rt_ws_bytes(int, int, int, int, const tp_rtsvd_params*, bool);
template <typename T>
tp_status rt_solve(const T*, const T*, const T*, int, int, int, int, const tp_rtsvd_params*, T*, tp_info*, void*,
                   size_t, cudaStream_t, int, const void*);
template <typename T>
tp_status rt_adjoint(const T*, int, int, int, int, const tp_rtsvd_params*, T*, void*, size_t, cudaStream_t);
template <typename T> size_t tt_ws_bytes(int, int, int, int, const tp_ttsvd_params*);
template <typename T>
tp_status tt_adjoint(const T*, int, int, int, int, const tp_ttsvd_params*, T*, void*, size_t, cudaStream_t);
template <typename T>
tp_status tt_solve(const T*, const T*, int, int, int, int, const tp_ttsvd_params*, T*, tp_info*, void*, size_t,
                   cudaStream_t);
template <typename T> size_t gk_ws_bytes(int, int, int, int, const tp_tgkb_params*);
template <typename T>
tp_status gk_solve(const T*, const T*, int, int, int, int, const tp_tgkb_params*, T*, tp_info*, void*, size_t,
                   cudaStream_t, const void*);
template <typename T> size_t gkn_ws_bytes(int, int, int, int, const tp_tgkb_params*);
template <typename T>
tp_status gkn_solve(const T*, const T*, int, int, int, int, const tp_tgkb_params*, T*, tp_info*, void*, size_t,
                    cudaStream_t);
template <typename T> size_t tri_ws_bytes(int, int, int, int);
template <typename T>
tp_status tri_solve(const T*, const T*, int, int, int, int, T*, T*, T*, void*, size_t, cudaStream_t);
template <typename T> size_t tik_ws_bytes(int, int, int, int, const tp_tik_params*);
template <typename T>
tp_status tik_solve(const T*, const T*, int, int, int, int, const tp_tik_params*, T*, tp_info*, void*, size_t,
                    cudaStream_t, const void*);

static bool dims_ok(int l, int m, int n, int prec) {
    if (l < 1 || m < 1 || n < 1) return false;
    if (prec != TP_FP32 && prec != TP_FP64) return false;
    if (n > (prec == TP_FP32 ? 1024 : 512)) return false;
    return (long)l * m * n < (1L << 40);
}

template <typename T>
static tp_status fft_t(const void* A, int l, int m, int n, void* Ahat, cudaStream_t st) {
    return rdft<T>((const T*)A, Ahat, n, l, m, m, (long)l * m, nullptr, nullptr, st);
}
template <typename T>
static tp_status ifft_t(const void* Xh, int l, int m, int n, void* X, cudaStream_t st) {
    return irdft<T>(Xh, (T*)X, n, l, m, m, (long)l * m, nullptr, st);
}

static size_t gemm_ws(int l, int kk, int m, int n, size_t c) {
    const size_t h = n / 2 + 1;
    return align256(h * l * kk * c) + align256(h * kk * m * c) + align256(h * l * m * c);
}

template <typename T>
static tp_status gemm_t(const void* A, const void* B, void* C, int l, int kk, int m, int n, int trans, void* ws,
                        cudaStream_t st, int tc_passes = 3) {
    const int h = n / 2 + 1;
    const size_t c = 2 * sizeof(T);
    char* p = (char*)ws;
    void* Ah = p;
    void* Bh = p + align256((size_t)h * l * kk * c);
    void* Ch = (char*)Bh + align256((size_t)h * kk * m * c);
    // A is (n, l, kk) or, t-transposed, (n, kk, l); B is (n, kk, m) or (n, m, kk).
    // The t-transpose is the conjugate transpose of every Fourier slice.
    const bool tA = trans & 1, tB = trans & 2;
    const int ar = tA ? kk : l, ac = tA ? l : kk;
    const int br = tB ? m : kk, bc = tB ? kk : m;
    tp_status e = rdft<T>((const T*)A, Ah, n, ar, ac, ac, (long)ar * ac, nullptr, nullptr, st);
    if (e != TP_OK) return e;
    e = rdft<T>((const T*)B, Bh, n, br, bc, bc, (long)br * bc, nullptr, nullptr, st);
    if (e != TP_OK) return e;
    e = cgemm<T>(h, l, m, kk, nullptr, nullptr, nullptr, 1, 0, Ah, ac, (long)ar * ac, tA ? OP_C : OP_N, Bh, bc,
                 (long)br * bc, tB ? OP_C : OP_N, 0, 0, Ch, m, (long)l * m, nullptr, st, nullptr, tc_passes);
    if (e != TP_OK) return e;
    return irdft<T>(Ch, (T*)C, n, l, m, m, (long)l * m, nullptr, st);
}

}  // namespace tp

using namespace tp;

extern "C" {

tp_status tprod_fft(const void* A, int l, int m, int n, void* Ahat, int prec, void* stream) {
    if (!A || !Ahat || !dims_ok(l, m, n, prec)) return TP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    return prec == TP_FP32 ? fft_t<float>(A, l, m, n, Ahat, st) : fft_t<double>(A, l, m, n, Ahat, st);
}

tp_status tprod_ifft(const void* Xhat, int l, int m, int n, void* X, int prec, void* stream) {
    if (!Xhat || !X || !dims_ok(l, m, n, prec)) return TP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    return prec == TP_FP32 ? ifft_t<float>(Xhat, l, m, n, X, st) : ifft_t<double>(Xhat, l, m, n, X, st);
}

// TP_TF32: float32 data; only the tensor-core products differ (one tf32 product).
static int data_prec(int prec) { return prec == TP_TF32 ? TP_FP32 : prec; }

size_t tprod_gemm_workspace_bytes(int l, int kk, int m, int n, int prec) {
    prec = data_prec(prec);
    if (!dims_ok(l, kk, n, prec) || m < 1) return 0;
    return gemm_ws(l, kk, m, n, prec == TP_FP32 ? 8 : 16);
}

tp_status tprod_gemm(const void* A, const void* B, void* C, int l, int kk, int m, int n, int trans, int prec,
                     void* ws, size_t ws_bytes, void* stream) {
    const int passes = prec == TP_TF32 ? 1 : 3;
    prec = data_prec(prec);
    if (!A || !B || !C || !dims_ok(l, kk, n, prec) || !dims_ok(kk, m, n, prec)) return TP_ERR_ARG;
    if (trans < 0 || trans > 3) return TP_ERR_ARG;
    if (l > 65535 * 128) return TP_ERR_ARG;
    const size_t need = gemm_ws(l, kk, m, n, prec == TP_FP32 ? 8 : 16);
    if (!ws || ((size_t)ws & 255) || ws_bytes < need) return TP_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    return prec == TP_FP32 ? gemm_t<float>(A, B, C, l, kk, m, n, trans, ws, st, passes)
                           : gemm_t<double>(A, B, C, l, kk, m, n, trans, ws, st);
}

size_t rtsvd_workspace_bytes(int l, int m, int n, int p, const tp_rtsvd_params* params, int prec) {
    prec = data_prec(prec);
    if (prec == TP_BF16) return rt_ws_bytes<float>(l, m, n, p, params, true);
    if (prec == TP_FP32) return rt_ws_bytes<float>(l, m, n, p, params, false);
    if (prec == TP_FP64) return rt_ws_bytes<double>(l, m, n, p, params, false);
    return 0;
}

tp_status rtsvd_truncated_solve(const void* A, const void* B, const void* Omega, int l, int m, int n, int p,
                                const tp_rtsvd_params* params, void* X, tp_info* d_info, int prec, void* ws,
                                size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == TP_FP32 || prec == TP_TF32 || prec == TP_BF16)
        return rt_solve<float>((const float*)A, (const float*)B, (const float*)Omega, l, m, n, p, params, (float*)X,
                               d_info, ws, ws_bytes, st, prec == TP_TF32 ? 1 : (prec == TP_BF16 ? 0 : 3), nullptr);
    if (prec == TP_FP64)
        return rt_solve<double>((const double*)A, (const double*)B, (const double*)Omega, l, m, n, p, params,
                                (double*)X, d_info, ws, ws_bytes, st, 3, nullptr);
    return TP_ERR_ARG;
}


tp_status rtsvd_truncated_solve_hat(const void* Ahat, const void* B, const void* Omega, int l, int m, int n, int p,
                                    const tp_rtsvd_params* params, void* X, tp_info* d_info, int prec, void* ws,
                                    size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!Ahat) return TP_ERR_ARG;
    if (prec == TP_FP32 || prec == TP_TF32 || prec == TP_BF16)
        return rt_solve<float>(nullptr, (const float*)B, (const float*)Omega, l, m, n, p, params, (float*)X, d_info,
                               ws, ws_bytes, st, prec == TP_TF32 ? 1 : (prec == TP_BF16 ? 0 : 3), Ahat);
    if (prec == TP_FP64)
        return rt_solve<double>(nullptr, (const double*)B, (const double*)Omega, l, m, n, p, params, (double*)X,
                                d_info, ws, ws_bytes, st, 3, Ahat);
    return TP_ERR_ARG;
}

tp_status rtsvd_adjoint(const void* G, int l, int m, int n, int p, const tp_rtsvd_params* params, void* dB,
                        int prec, void* ws, size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == TP_FP32 || prec == TP_TF32)
        return rt_adjoint<float>((const float*)G, l, m, n, p, params, (float*)dB, ws, ws_bytes, st);
    if (prec == TP_FP64) return rt_adjoint<double>((const double*)G, l, m, n, p, params, (double*)dB, ws, ws_bytes, st);
    return TP_ERR_ARG;
}

tp_status ttsvd_adjoint(const void* G, int l, int m, int n, int p, const tp_ttsvd_params* params, void* dB, int prec,
                        void* ws, size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == TP_FP32) return tt_adjoint<float>((const float*)G, l, m, n, p, params, (float*)dB, ws, ws_bytes, st);
    if (prec == TP_FP64)
        return tt_adjoint<double>((const double*)G, l, m, n, p, params, (double*)dB, ws, ws_bytes, st);
    return TP_ERR_ARG;
}

size_t ttsvd_workspace_bytes(int l, int m, int n, int p, const tp_ttsvd_params* params, int prec) {
    if (prec == TP_FP32) return tt_ws_bytes<float>(l, m, n, p, params);
    if (prec == TP_FP64) return tt_ws_bytes<double>(l, m, n, p, params);
    return 0;
}

tp_status ttsvd_solve(const void* A, const void* B, int l, int m, int n, int p, const tp_ttsvd_params* params,
                      void* X, tp_info* d_info, int prec, void* ws, size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == TP_FP32)
        return tt_solve<float>((const float*)A, (const float*)B, l, m, n, p, params, (float*)X, d_info, ws, ws_bytes,
                               st);
    if (prec == TP_FP64)
        return tt_solve<double>((const double*)A, (const double*)B, l, m, n, p, params, (double*)X, d_info, ws,
                                ws_bytes, st);
    return TP_ERR_ARG;
}

size_t tgkb_workspace_bytes(int l, int m, int n, int p, const tp_tgkb_params* params, int prec) {
    if (prec == TP_FP32) return gk_ws_bytes<float>(l, m, n, p, params);
    if (prec == TP_FP64) return gk_ws_bytes<double>(l, m, n, p, params);
    return 0;
}

tp_status tgkb_solve(const void* A, const void* B, int l, int m, int n, int p, const tp_tgkb_params* params, void* X,
                     tp_info* d_info, int prec, void* ws, size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == TP_FP32)
        return gk_solve<float>((const float*)A, (const float*)B, l, m, n, p, params, (float*)X, d_info, ws, ws_bytes,
                               st, nullptr);
    if (prec == TP_FP64)
        return gk_solve<double>((const double*)A, (const double*)B, l, m, n, p, params, (double*)X, d_info, ws,
                                ws_bytes, st, nullptr);
    return TP_ERR_ARG;
}

tp_status tgkb_solve_hat(const void* Ahat, const void* B, int l, int m, int n, int p, const tp_tgkb_params* params,
                         void* X, tp_info* d_info, int prec, void* ws, size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!Ahat) return TP_ERR_ARG;
    if (prec == TP_FP32)
        return gk_solve<float>(nullptr, (const float*)B, l, m, n, p, params, (float*)X, d_info, ws, ws_bytes, st,
                               Ahat);
    if (prec == TP_FP64)
        return gk_solve<double>(nullptr, (const double*)B, l, m, n, p, params, (double*)X, d_info, ws, ws_bytes, st,
                                Ahat);
    return TP_ERR_ARG;
}

size_t nested_tgkb_workspace_bytes(int l, int m, int n, int p, const tp_tgkb_params* params, int prec) {
    if (prec == TP_FP32) return gkn_ws_bytes<float>(l, m, n, p, params);
    if (prec == TP_FP64) return gkn_ws_bytes<double>(l, m, n, p, params);
    return 0;
}

tp_status nested_tgkb_solve(const void* A, const void* B, int l, int m, int n, int p, const tp_tgkb_params* params,
                            void* X, tp_info* d_info, int prec, void* ws, size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == TP_FP32)
        return gkn_solve<float>((const float*)A, (const float*)B, l, m, n, p, params, (float*)X, d_info, ws, ws_bytes,
                                st);
    if (prec == TP_FP64)
        return gkn_solve<double>((const double*)A, (const double*)B, l, m, n, p, params, (double*)X, d_info, ws,
                                 ws_bytes, st);
    return TP_ERR_ARG;
}

size_t tgkb_triplets_workspace_bytes(int l, int m, int n, int k, int prec) {
    if (prec == TP_FP32) return tri_ws_bytes<float>(l, m, n, k);
    if (prec == TP_FP64) return tri_ws_bytes<double>(l, m, n, k);
    return 0;
}

tp_status tgkb_triplets(const void* A, const void* B, int l, int m, int n, int k, void* U, void* S, void* V, int prec,
                        void* ws, size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == TP_FP32)
        return tri_solve<float>((const float*)A, (const float*)B, l, m, n, k, (float*)U, (float*)S, (float*)V, ws,
                                ws_bytes, st);
    if (prec == TP_FP64)
        return tri_solve<double>((const double*)A, (const double*)B, l, m, n, k, (double*)U, (double*)S, (double*)V,
                                 ws, ws_bytes, st);
    return TP_ERR_ARG;
}

size_t tgkb_tikhonov_workspace_bytes(int l, int m, int n, int p, const tp_tik_params* params, int prec) {
    if (prec == TP_FP32) return tik_ws_bytes<float>(l, m, n, p, params);
    if (prec == TP_FP64) return tik_ws_bytes<double>(l, m, n, p, params);
    return 0;
}

tp_status tgkb_tikhonov_solve(const void* A, const void* B, int l, int m, int n, int p, const tp_tik_params* params,
                              void* X, tp_info* d_info, int prec, void* ws, size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == TP_FP32)
        return tik_solve<float>((const float*)A, (const float*)B, l, m, n, p, params, (float*)X, d_info, ws,
                                ws_bytes, st, nullptr);
    if (prec == TP_FP64)
        return tik_solve<double>((const double*)A, (const double*)B, l, m, n, p, params, (double*)X, d_info, ws,
                                 ws_bytes, st, nullptr);
    return TP_ERR_ARG;
}

tp_status tgkb_tikhonov_solve_hat(const void* Ahat, const void* B, int l, int m, int n, int p,
                                  const tp_tik_params* params, void* X, tp_info* d_info, int prec, void* ws,
                                  size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!Ahat) return TP_ERR_ARG;
    if (prec == TP_FP32)
        return tik_solve<float>(nullptr, (const float*)B, l, m, n, p, params, (float*)X, d_info, ws, ws_bytes, st,
                                Ahat);
    if (prec == TP_FP64)
        return tik_solve<double>(nullptr, (const double*)B, l, m, n, p, params, (double*)X, d_info, ws, ws_bytes, st,
                                 Ahat);
    return TP_ERR_ARG;
}

tp_status sep_operator(const void* T, const double* c, int l, int m, int n, void* A, int prec, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == TP_FP32) return sep_operator<float>((const float*)T, c, l, m, n, (float*)A, st);
    if (prec == TP_FP64) return sep_operator<double>((const double*)T, c, l, m, n, (double*)A, st);
    return TP_ERR_ARG;
}

size_t sep_grad_c_workspace_bytes(int m, int n, int p, int prec) {
    if (prec == TP_FP32) return sep_ws_bytes<float>(m, n, p);
    if (prec == TP_FP64) return sep_ws_bytes<double>(m, n, p);
    return 0;
}

tp_status sep_grad_c(const void* X, const void* G, const double* c, int m, int n, int p, double* dc, int prec,
                     void* ws, size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == TP_FP32)
        return sep_grad<float>((const float*)X, (const float*)G, c, m, n, p, dc, ws, ws_bytes, st);
    if (prec == TP_FP64)
        return sep_grad<double>((const double*)X, (const double*)G, c, m, n, p, dc, ws, ws_bytes, st);
    return TP_ERR_ARG;
}

size_t tgkb_tikhonov_grad_c_workspace_bytes(int l, int m, int n, const tp_tik_params* params, int prec) {
    if (prec == TP_FP32) return tik_grad_ws_bytes<float>(l, m, n, params);
    if (prec == TP_FP64) return tik_grad_ws_bytes<double>(l, m, n, params);
    return 0;
}

tp_status tgkb_tikhonov_grad_c(const void* G, const double* c, int l, int m, int n, const tp_tik_params* params,
                               const void* solve_ws, size_t solve_ws_bytes, double* dc, int prec, void* ws,
                               size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == TP_FP32)
        return tik_grad_c<float>((const float*)G, c, l, m, n, params, solve_ws, solve_ws_bytes, dc, ws, ws_bytes,
                                 st);
    if (prec == TP_FP64)
        return tik_grad_c<double>((const double*)G, c, l, m, n, params, solve_ws, solve_ws_bytes, dc, ws,
                                  ws_bytes, st);
    return TP_ERR_ARG;
}

size_t tgkb_adjoint_workspace_bytes(int l, int m, int n, const tp_tgkb_params* params, int prec) {
    if (prec == TP_FP32) return gk_adj_ws_bytes<float>(l, m, n, params);
    if (prec == TP_FP64) return gk_adj_ws_bytes<double>(l, m, n, params);
    return 0;
}

tp_status tgkb_adjoint(const void* G, int l, int m, int n, const tp_tgkb_params* params, const void* solve_ws,
                       size_t solve_ws_bytes, const void* Ahat, void* dB, int prec, void* ws, size_t ws_bytes,
                       void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == TP_FP32)
        return gk_adjoint<float>((const float*)G, l, m, n, params, solve_ws, solve_ws_bytes, Ahat, (float*)dB, ws,
                                 ws_bytes, st);
    if (prec == TP_FP64)
        return gk_adjoint<double>((const double*)G, l, m, n, params, solve_ws, solve_ws_bytes, Ahat, (double*)dB,
                                  ws, ws_bytes, st);
    return TP_ERR_ARG;
}

size_t tgkb_tikhonov_adjoint_workspace_bytes(int l, int m, int n, const tp_tik_params* params, int prec) {
    if (prec == TP_FP32) return tik_adj_ws_bytes<float>(l, m, n, params);
    if (prec == TP_FP64) return tik_adj_ws_bytes<double>(l, m, n, params);
    return 0;
}

tp_status tgkb_tikhonov_adjoint(const void* G, int l, int m, int n, const tp_tik_params* params, const void* solve_ws,
                                size_t solve_ws_bytes, const void* Ahat, void* dB, int prec, void* ws,
                                size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == TP_FP32)
        return tik_adjoint<float>((const float*)G, l, m, n, params, solve_ws, solve_ws_bytes, Ahat, (float*)dB, ws,
                                  ws_bytes, st);
    if (prec == TP_FP64)
        return tik_adjoint<double>((const double*)G, l, m, n, params, solve_ws, solve_ws_bytes, Ahat, (double*)dB,
                                   ws, ws_bytes, st);
    return TP_ERR_ARG;
}

tp_status rtsvd_autotune(int l, int m, int n, int p, const tp_rtsvd_params* params, int prec, void* ws,
                         size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!params || l < 1 || m < 1 || n < 1 || p < 1 || params->block < 1 || params->r_max < 1) return TP_ERR_ARG;
    if (prec == TP_FP64) return TP_OK;  // the float64 products run on the SIMT kernel: nothing to tune
    if (prec != TP_FP32 && prec != TP_TF32 && prec != TP_BF16) return TP_ERR_ARG;
    if (!ws || ((uintptr_t)ws & 255)) return TP_ERR_WORKSPACE;
    const int h = n / 2 + 1, b = params->block < params->r_max ? params->block : params->r_max;
    const int sk = prec == TP_FP32 ? 3 : (prec == TP_TF32 ? 1 : 0);
    // the products of a solve: sketch A-hat Omega_b and the power iteration's A-hat Z (op N), A-hat^H Y from
    // the transposed copy (op R) in the sketch precision, the re-projection A-hat^H Y (float32-accurate) and
    // the column chunks of K = A-hat V (float32-accurate, 32 columns, written transposed)
    struct Shape { int op, M, N, K, passes, trans; } shapes[4] = {
        {OP_N, l, b, m, sk, 0}, {OP_R, m, b, l, sk, 0}, {OP_R, m, b, l, 3, 0},
        {OP_N, l, params->r_max < 32 ? params->r_max : 32, m, 3, 1}};
    for (const Shape& sh : shapes) {
        if (sh.passes == 0 && ((l & 3) || (m & 3))) continue;  // the BF16 form refuses these shapes
        const tp_status e = zgemm_tc_tune(h, sh.M, sh.N, sh.K, sh.op, sh.passes, sh.trans, ws, ws_bytes, st, nullptr,
                                          nullptr, nullptr);
        if (e != TP_OK && e != TP_ERR_UNSUPPORTED) return e;
    }
    return TP_OK;
}

int tp_autotune_table(int* ints, float* flts, int max) {
    if (!ints || !flts || max < 0) return 0;
    return zgemm_tc_tuned(ints, flts, max);
}

void tp_autotune_clear(void) { zgemm_tc_untune(); }

tp_status tp_autotune_set(int op, int passes, int columns, int M, int K, int batch, int stages) {
    if ((op != OP_N && op != OP_R && op != OP_C) || (passes != 0 && passes != 1 && passes != 3) || columns < 1 ||
        columns > 32 || M < 1 || K < 1 || batch < 1)
        return TP_ERR_ARG;
    return zgemm_tc_set(op, passes, columns, M, K, batch, stages) == TP_OK ? TP_OK : TP_ERR_ARG;
}

const char* tp_status_string(int status) {
    switch (status) {
        case TP_OK: return "ok";
        case TP_ERR_ARG: return "invalid argument";
        case TP_ERR_CUDA: return "CUDA launch or attribute call failed";
        case TP_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case TP_ERR_BREAKDOWN: return "breakdown";
        case TP_ERR_NOT_CONVERGED: return "discrepancy principle not met within the cap";
        case TP_ERR_TIMEOUT: return "bounded device-side wait gave up";
        case TP_ERR_UNSUPPORTED: return "request not supported by this build or device";
        case TP_ERR_NONFINITE: return "input holds a NaN or an infinity";
        default: return "unknown status";
    }
}

int tp_version(void) { return 100; }

int tp_kernel_launches(void) { return g_launches; }

int tp_wait_budget(long long cycles) {
    if (cycles < 0) return TP_ERR_ARG;
    tp::g_wait_budget.store(cycles);
    return TP_OK;
}

int tp_wait_stall(int on) {
    if (on != 0 && on != 1) return TP_ERR_ARG;
    tp::g_wait_stall.store(on);
    return TP_OK;
}

int tp_timing_enable(int class_mask) {
    g_mask = class_mask & ((1 << TP_KC_COUNT) - 1);
    return TP_OK;
}

int tp_timing_read(double* ms, int* launches, int nclasses) {
    if (!ms || !launches || nclasses < 1) return TP_ERR_ARG;
    for (int c = 0; c < nclasses; ++c) {
        ms[c] = 0.0;
        launches[c] = 0;
    }
    int rc = TP_KC_COUNT;
    for (const Rec& r : g_recs) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
            rc = TP_ERR_CUDA;
        if (r.cls < nclasses) {
            ms[r.cls] += t;
            launches[r.cls] += 1;
        }
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    return rc;
}

}  // extern "C"
