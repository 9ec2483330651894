// tprod_gemm_noalloc: the t-product of tprod_gemm computed in a fixed scratch
// array that the library owns, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// that runs inside a host framework whose device memory is owned by an
// allocator it cannot reach (plugins, language bindings without a CUDA
// allocator), and latency-critical paths whose rules forbid allocation after
// start-up because cudaMalloc can block and synchronise the device.  This
// entry point needs nothing from them but inputs and outputs.
//
// The scratch is one static device array of NOALLOC_SCRATCH_BYTES (16 MiB).
// Every GPU on which the library is loaded holds that array until the
// process exits.  Problems whose three spectra (A-hat, B-hat, C-hat) do not
// fit are rejected with TP_ERR_WORKSPACE before anything is enqueued.
//
// In host code the array's name is only a host-side stand-in for the device
// symbol, so its device address is looked up with cudaGetSymbolAddress once
// per device, with that device current, the first time the entry point runs
// there.  Make that first call on each device before any stream capture.
//
// All calls share the one array and every call overwrites the parts it uses
// (the transforms and the product write every element they later read), so
// nothing needs clearing between calls; but two calls whose work overlaps on
// the GPU (different streams, or different host threads) race on the array.
#include <mutex>

#include "common.cuh"
#include "internal.h"

static constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

tp_status scratch_for_current_device(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return TP_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return TP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();  // leave no stale error for the next call on this thread
            return TP_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return TP_OK;
}

template <typename T>
tp_status run(const void* A, const void* B, void* C, int l, int kk, int m, int n, int transA, char* ws,
              cudaStream_t st) {
    using namespace tp;
    const int h = n / 2 + 1;
    const size_t c = 2 * sizeof(T);
    void* Ah = ws;
    void* Bh = ws + align256((size_t)h * l * kk * c);
    void* Ch = (char*)Bh + align256((size_t)h * kk * m * c);
    const int ar = transA ? kk : l, ac = transA ? l : kk;
    tp_status e = rdft<T>((const T*)A, Ah, n, ar, ac, ac, (long)ar * ac, nullptr, nullptr, st);
    if (e != TP_OK) return e;
    e = rdft<T>((const T*)B, Bh, n, kk, m, m, (long)kk * m, nullptr, nullptr, st);
    if (e != TP_OK) return e;
    e = cgemm<T>(h, l, m, kk, nullptr, nullptr, nullptr, 1, 0, Ah, ac, (long)ar * ac, transA ? OP_C : OP_N, Bh, m,
                 (long)kk * m, OP_N, 0, 0, Ch, m, (long)l * m, nullptr, st);
    if (e != TP_OK) return e;
    return irdft<T>(Ch, (T*)C, n, l, m, m, (long)l * m, nullptr, st);
}

}  // namespace

extern "C" tp_status tprod_gemm_noalloc(const void* A, const void* B, void* C, int l, int kk, int m, int n,
                                        int transA, int prec, void* stream) {
    if (!A || !B || !C || l < 1 || kk < 1 || m < 1 || n < 1) return TP_ERR_ARG;
    if (prec != TP_FP32 && prec != TP_FP64) return TP_ERR_ARG;
    if (transA != 0 && transA != 1) return TP_ERR_ARG;
    if (n > (prec == TP_FP32 ? 1024 : 512)) return TP_ERR_ARG;
    // the size limits of tprod_gemm: with every operand below 2^40 elements the
    // byte counts below cannot wrap
    const long lim = 1L << 40;
    if ((long)l * kk * n >= lim || (long)kk * m * n >= lim || (long)l * m * n >= lim) return TP_ERR_ARG;
    if (l > 65535 * 128) return TP_ERR_ARG;
    const size_t c = prec == TP_FP32 ? 8 : 16;
    const size_t h = (size_t)n / 2 + 1;
    const size_t need = tp::align256(h * l * kk * c) + tp::align256(h * kk * m * c) + tp::align256(h * l * m * c);
    if (need > NOALLOC_SCRATCH_BYTES) return TP_ERR_WORKSPACE;
    void* ws = nullptr;
    const tp_status e = scratch_for_current_device(&ws);
    if (e != TP_OK) return e;
    cudaStream_t st = (cudaStream_t)stream;
    return prec == TP_FP32 ? run<float>(A, B, C, l, kk, m, n, transA, (char*)ws, st)
                           : run<double>(A, B, C, l, kk, m, n, transA, (char*)ws, st);
}
