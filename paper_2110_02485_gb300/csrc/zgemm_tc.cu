// Batched complex matrix product C[s] = op(A[s]) B[s] on the fifth-generation
// tensor cores (tcgen05.mma, kind::tf32) with float32 accuracy.
//
// This is the sketch and projection product of the block RT-tSVD (Algorithm 3
// in block form: Y = A-hat Omega-hat, Z = A-hat^H Y per Fourier slice), whose
// right-hand side has few columns (the block size b <= 32) while A-hat is a
// full slice.  The complex product is written as a real one:
//   op = N:  rows i of A, reduction over (j, re/im), A used in place;
//   op = C:  rows (j, re/im) of A^T, reduction over i, A transposed while it
//            is staged in shared memory,
// with the right-hand side expanded into a real matrix of 2 b columns whose
// signs produce the real and imaginary parts (conjugation included).
//
// Accuracy: each float32 operand x is split as x = hi + lo and the product
// keeps hi*hi + hi*lo + lo*hi (the "3xTF32" scheme).  The tensor core reads a
// float32 operand as tf32 by ignoring its 13 low mantissa bits, so for the
// large operand (A) with op = N or R hi is the float32 tile itself, left in
// place, and lo = x - trunc(x) (read as tf32, i.e. truncated) is the only
// value written; otherwise hi = rna(x), lo = rna(x - hi).  Relative error of
// a term: at most about 2^-20, the order of float32 products.  The right-hand
// side's hi and lo rows are stacked, so one MMA of N = 4 b' forms hi*hi and
// hi*lo and a second of N = 2 b' adds lo*hi (b' = b rounded up to 8).
//
// Layout and pipeline: one CTA per (slice, 128-row tile), three roles that
// meet only at mbarriers, over a ring of stages:
//   warp 8 (one thread): TMA loads of the raw A and B tiles of a stage
//        (3-D tensor maps: columns, rows, slices; zero fill past the edges);
//   warps 0-7: the hi/lo split.  For op = N the TMA writes A with the 128-byte
//        swizzle, which is the tensor core's K-major SWIZZLE_128B layout, so
//        hi is the tile in place and lo is written to tensor memory (one lane
//        per row; the lo*hi MMA reads its A operand from there); for op = C the
//        raw tile (rows i) is transposed into the no-swizzle K-major layout
//        (8 rows x 16 bytes per core matrix).  The real right-hand side is
//        built from the raw B rows;
//   warp 9 (one thread): the MMAs of a stage, committed to the stage's
//        "empty" barrier, which hands the buffers back to the TMA thread.
// The accumulator (128 lanes x 4 b' float32 columns) lives in tensor memory,
// followed by the lo tiles of the stages (op = N, 3xTF32);
// warps 0-7 read it back with tcgen05.ld once the last commit lands.
// op = R (conj(A) B, A row-major) uses the op = N kernel with the signs of
// the right-hand side flipped; the RT-tSVD forms A-hat^H Y this way from a
// transposed copy of A-hat, so every large product takes the swizzled path.
// BF16 form (NP = 0): A is a bfloat16 copy of the complex matrix (interleaved
// re, im; 4 bytes per entry), the right-hand side is rounded to bfloat16 as it
// is expanded, and the MMAs are kind::f16 with float32 accumulation: a stage
// holds 64 real reduction entries (the same 128-byte swizzled rows), one MMA
// per 16-entry step, no lo tile.  Relative error of a product term about 2^-8.
// Every wait is bounded; on a timeout the kernel records TP_ERR_TIMEOUT,
// waits (bounded) for its MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "internal.h"

namespace tp {
namespace {

constexpr int TC_M = 128;                 // MMA rows per CTA
constexpr int TC_KT = 32;                 // real reduction length per stage (4 MMA K-steps of 8)
constexpr int TC_CONV_WARPS = 8;          // warps 0-7 split; in the epilogue warp w reads TMEM lanes 32 (w % 4)..
constexpr int TC_CONV_THREADS = 32 * TC_CONV_WARPS;
constexpr int TC_PROD_WARP = TC_CONV_WARPS, TC_MMA_WARP = TC_CONV_WARPS + 1;
constexpr int TC_THREADS = 32 * (TC_CONV_WARPS + 2);
constexpr int TC_A_BYTES = TC_M * TC_KT * 4;      // one A tile (16 KB)
constexpr uint32_t TC_LBO_A = (TC_M / 8) * 128;  // no-swizzle K-major: next core matrix along K
constexpr uint32_t TC_SBO = 128;                  // no-swizzle: next core matrix along M / N
constexpr uint32_t TC_SBO_SW = 1024;              // 128-byte swizzle: next 8-row group
constexpr int TC_SMEM_LIMIT = 225 * 1024;
constexpr long long TC_SPIN = 2000000000LL;       // ~1 s at the GB300 SM clock
constexpr int TC_NS_CAP = 6;                      // stages of the ring at most (barrier arrays)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// x rounded to tf32 (10 stored mantissa bits), to nearest with ties away from
// zero: add half an ulp of the kept part to the magnitude bits, clear the rest
// (a carry into the exponent is the correct rounding; finite inputs only).
__device__ __forceinline__ float tf32_rna(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void split3(float x, float& hi, float& lo) {
    hi = tf32_rna(x);
    lo = tf32_rna(x - hi);
}
__device__ __forceinline__ void split3(float4 x, float4& hi, float4& lo) {
    split3(x.x, hi.x, lo.x);
    split3(x.y, hi.y, lo.y);
    split3(x.z, hi.z, lo.z);
    split3(x.w, hi.w, lo.w);
}
// The part of x below its tf32 truncation (exact in float32).  It is left
// unrounded: the tensor core reads it as tf32 by dropping its low bits, an
// error of at most 2^-20 |x|, the size of the lo*lo term the split already
// neglects (an emulation of the product over Gaussian data: 7.7e-9 mean and
// 3.9e-8 largest error relative to |A||B|, against 6.0e-9 and 3.4e-8 with lo
// rounded to nearest).
__device__ __forceinline__ float tf32_rest(float x) {
    return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, descriptor version 1, layout type (0 none, 2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout = 0) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)layout << 61);
}
// Instruction descriptor, kind::tf32: D float32, A and B tf32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Instruction descriptor, kind::f16: D float32, A and B bfloat16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// A from tensor memory (columns of one lane per row), B from shared memory.
__device__ __forceinline__ void mma_tf32_ta(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}"
        :
        : "r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity (at most `spin` cycles).
// False on timeout (which also raises *abort) or when another role has raised
// *abort.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort, long long spin) {
    const long long t0 = clock64();
    while (!mbar_try(a, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > spin) {
            *abort = 1;
            return false;
        }
    }
    return true;
}
// Bounded wait that ignores the abort flag (used to drain work in flight: TMA
// writes and MMAs already issued, which complete whatever the other roles do;
// its bound is fixed, never the progress budget).
__device__ __forceinline__ void mbar_drain(uint32_t a, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try(a, parity))
        if (clock64() - t0 > TC_SPIN) return;
}
__device__ __forceinline__ void mbar_init_n(uint32_t a, unsigned n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8 consecutive float32 columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    // the registers are valid only after wait::ld; threading them through the
    // wait keeps every use behind it
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive 32-bit columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Byte offset of element (row, k) in a K-major no-swizzle tile whose core
// matrices advance by `lbo` along K and by 128 bytes along the rows.
__device__ __forceinline__ uint32_t kmaj_off(int row, int k, uint32_t lbo) {
    return (uint32_t)(k >> 2) * lbo + (uint32_t)(row >> 3) * TC_SBO + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

// The same for 2-byte elements: 8 per 16-byte core-matrix row.
__device__ __forceinline__ uint32_t kmaj_off16(int row, int k, uint32_t lbo) {
    return (uint32_t)(k >> 3) * lbo + (uint32_t)(row >> 3) * TC_SBO + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ float pick4(const float4& v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

// Stage buffers: raw A (TMA), hi A (op C only; op N uses the raw tile), lo A
// (3xTF32 with op C only), raw B rows (TMA), and the real right-hand side
// B_op.  NP = 3 (hi*hi + hi*lo + lo*hi, float32 accuracy), 1 (hi*hi, the TF32
// precision form) or 0 (bfloat16 A and B_op, the BF16 form; op N only).  KT
// real reduction entries per stage: 32 in tf32, 64 in bfloat16 (the same
// 128-byte rows).  With op N and NP = 3 (LO_TM) the lo tile of A lives in
// tensor memory instead (32 columns per stage after the accumulator's, one
// lane per row), which is what the MMA's A operand may also be read from:
// a stage then takes 16 KB less shared memory, so two CTAs per SM keep four
// tiles each in flight.
template <int OPA, int NCP, int NP> struct TcCfg {
    static constexpr int KT = NP == 0 ? 2 * TC_KT : TC_KT;
    static constexpr int NB = (NP == 3 ? 4 : 2) * NCP;  // B_op rows: (re, im) x (hi[, lo])
    static constexpr bool LO_TM = NP == 3 && OPA == OP_N;
    static constexpr uint32_t LBO_B = (NB / 8) * 128;
    static constexpr int KB = OPA == OP_N ? KT / 2 : KT;  // B rows per stage
    static constexpr int A_RAW = 0;
    static constexpr int A_HI = OPA == OP_N ? 0 : TC_A_BYTES;
    static constexpr int A_LO = A_HI + TC_A_BYTES;  // used when NP == 3 and not LO_TM
    static constexpr int B_RAW = (NP == 3 && !LO_TM ? A_LO : A_HI) + TC_A_BYTES;
    static constexpr int B_RAW_BYTES = KB * NCP * 8;
    static constexpr int B_OP = B_RAW + B_RAW_BYTES;
    static constexpr int STAGE = B_OP + NB * KT * (NP == 0 ? 2 : 4);
    static_assert(STAGE % 1024 == 0, "stages start on the 128-byte swizzle's 1024-byte period");
    // tensor-memory columns: the accumulator (NB, at least 32), then the lo tiles
    static constexpr int ACC = NB < 32 ? 32 : NB;
    static constexpr int tm_need(int ns) { return ACC + (LO_TM ? 32 * ns : 0); }
    // two CTAs per SM when two stages fit in half the shared memory (the TMA
    // stream of one CTA does not fill an SM's share of L2 bandwidth), with as
    // many stages as fit there (up to four: each CTA's tiles are latency-bound)
    // and in half the tensor memory, else one CTA with up to four stages
    static constexpr int NS2S = (TC_SMEM_LIMIT / 2 - 1024) / STAGE;
    static constexpr int NS2 = NS2S >= 2 && tm_need(NS2S > 4 ? 4 : NS2S) > 256 ? (256 - ACC) / 32 : NS2S;
    static constexpr int NS1 = (TC_SMEM_LIMIT - 1024) / STAGE >= 4 ? 4 : (TC_SMEM_LIMIT - 1024) / STAGE;
    static constexpr int NS = NS2 >= 2 ? (NS2 > 4 ? 4 : NS2) : NS1;
    // the most stages one CTA can hold (the autotuner's range is 2 .. NS_FIT)
    static constexpr int NSF_SM = (TC_SMEM_LIMIT - 1024) / STAGE > TC_NS_CAP ? TC_NS_CAP
                                                                            : (TC_SMEM_LIMIT - 1024) / STAGE;
    static constexpr int NS_FIT = tm_need(NSF_SM) > 512 ? (512 - ACC) / 32 : NSF_SM;
    // a stage count whose tensor memory exceeds half of it reserves more than
    // half the shared memory, so that a second CTA never waits in tcgen05.alloc
    static size_t smem(int ns) {
        const size_t s = (size_t)ns * STAGE + 1024;  // + alignment slack
        return tm_need(ns) > 256 && s <= (size_t)TC_SMEM_LIMIT / 2 ? (size_t)TC_SMEM_LIMIT / 2 + 1024 : s;
    }
    static constexpr uint32_t TX = TC_A_BYTES + B_RAW_BYTES;   // bytes the two TMA boxes deliver
    static uint32_t __host__ __device__ ncols(int ns) {       // power of two, at least 32
        uint32_t c = 32;
        while ((int)c < tm_need(ns)) c <<= 1;
        return c;
    }
};

// Split one stage (warps 0-7).  CONJ (op = R): right-hand side signs of conj(A) B.
// LO_TM: tlo is the tensor-memory address (lane 0) of this stage's lo tile.
template <int OPA, bool CONJ, int NCP, int NP>
__device__ __forceinline__ void split_stage(unsigned char* st, uint32_t tlo) {
    typedef TcCfg<OPA, NCP, NP> G;
    const int t = threadIdx.x;
    const float2* rb = (const float2*)(st + G::B_RAW);
    float* Bs = (float*)(st + G::B_OP);
    constexpr int RS = (NCP / 8) * TC_SBO;  // rows c, NCP + c, ...: NCP / 8 core matrices apart
    if (NP == 0) {
        // bfloat16: A is used as loaded; the right-hand side's re and im rows
        // (signs as below) rounded to bfloat16, two entries per 4-byte store
        const float sa = CONJ ? 1.f : -1.f, sb = CONJ ? -1.f : 1.f;
        for (int e = t; e < G::KB * NCP; e += TC_CONV_THREADS) {
            const int jj = e / NCP, c = e - jj * NCP;
            const float2 x = rb[e];
            char* q = (char*)Bs + kmaj_off16(c, 2 * jj, G::LBO_B);
            *(__nv_bfloat162*)(q) = __floats2bfloat162_rn(x.x, sa * x.y);
            *(__nv_bfloat162*)(q + RS) = __floats2bfloat162_rn(x.y, sb * x.x);
        }
        return;
    }
    if (OPA == OP_N) {
        if (NP == 3) {
            // hi is the swizzled tile itself; lo goes to tensor memory, one lane per
            // row: warp w takes rows 32 (w % 4) .. (its lanes) and reduction entries
            // 16 (w / 4) .. + 15, i.e. four 16-byte chunks of its row, chunk c of
            // row r sitting at chunk c ^ (r % 8) of the 128-byte line
            static_assert(TC_CONV_WARPS == 8 && TC_KT == 32, "two warps per lane quarter, 16 entries each");
            const int w = t >> 5, q = w & 3, hh = w >> 2, r = 32 * q + (t & 31);
            const unsigned char* row = st + G::A_RAW + (r >> 3) * 1024 + (r & 7) * 128;
            uint32_t v[16];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 x = *(const float4*)(row + (((4 * hh + j) ^ (r & 7)) << 4));
                v[4 * j] = __float_as_uint(tf32_rest(x.x));
                v[4 * j + 1] = __float_as_uint(tf32_rest(x.y));
                v[4 * j + 2] = __float_as_uint(tf32_rest(x.z));
                v[4 * j + 3] = __float_as_uint(tf32_rest(x.w));
            }
            tmem_st16(tlo + ((uint32_t)(32 * q) << 16) + 16u * hh, v);
        }
        // A B:       re row (Br, -Bi), im row (Bi,  Br)
        // conj(A) B: re row (Br,  Bi), im row (Bi, -Br)
        for (int e = t; e < G::KB * NCP; e += TC_CONV_THREADS) {
            const int jj = e / NCP, c = e - jj * NCP;
            const float2 x = rb[e];
            float rh, rl, ih, il;
            split3(x.x, rh, rl);
            split3(x.y, ih, il);
            const float sa = CONJ ? 1.f : -1.f, sb = CONJ ? -1.f : 1.f;
            char* p = (char*)Bs + kmaj_off(c, 2 * jj, G::LBO_B);
            *(float2*)(p) = make_float2(rh, sa * ih);
            *(float2*)(p + RS) = make_float2(ih, sb * rh);
            if (NP == 3) {
                *(float2*)(p + 2 * RS) = make_float2(rl, sa * il);
                *(float2*)(p + 3 * RS) = make_float2(il, sb * rl);
            }
        }
    } else {
        // raw rows i (128 floats each) -> rows (j, re/im) of the K-major tiles, 4 x 4 blocks
        const float* ra = (const float*)(st + G::A_RAW);
        float* Ahi = (float*)(st + G::A_HI);
        float* Alo = (float*)(st + G::A_LO);
#pragma unroll 1
        for (int b = t; b < (TC_M / 4) * (TC_KT / 4); b += TC_CONV_THREADS) {
            const int m4 = b & 31, i4 = b >> 5;
            float4 v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = *(const float4*)(ra + (4 * i4 + q) * 128 + 4 * m4);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = (u + (m4 >> 1)) & 3;  // rotate the first row with the thread: no bank conflicts
                const float4 w = make_float4(pick4(v[0], e), pick4(v[1], e), pick4(v[2], e), pick4(v[3], e));
                float4 hi, lo;
                split3(w, hi, lo);
                const uint32_t off = kmaj_off(4 * m4 + e, 4 * i4, TC_LBO_A);
                *(float4*)((char*)Ahi + off) = hi;
                if (NP == 3) *(float4*)((char*)Alo + off) = lo;
            }
        }
        for (int e = t; e < G::KB * NCP; e += TC_CONV_THREADS) {
            const int ii = e / NCP, c = e - ii * NCP;
            const float2 x = rb[e];
            float rh, rl, ih, il;
            split3(x.x, rh, rl);
            split3(x.y, ih, il);
            char* p = (char*)Bs + kmaj_off(c, ii, G::LBO_B);
            *(float*)(p) = rh;
            *(float*)(p + RS) = ih;
            if (NP == 3) {
                *(float*)(p + 2 * RS) = rl;
                *(float*)(p + 3 * RS) = il;
            }
        }
    }
}

template <int OPA, bool CONJ, int NCP, int NP>
__global__ void __launch_bounds__(TC_THREADS, 2)
k_zgemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
           float2* __restrict__ C, long ldc, long sC, int Mc, int Nc, int Kc, const int* skip, int* err,
           int trans_out, const int* ncap, int c0, long long spin, int ns) {
    typedef TcCfg<OPA, NCP, NP> G;
    if (skip && *skip) return;
    if (ncap && c0 >= *ncap) return;  // a column chunk past the run-time column count
    extern __shared__ unsigned char sm_raw[];
    __shared__ __align__(8) uint64_t full[TC_NS_CAP], conv[TC_NS_CAP], empty[TC_NS_CAP], accf;
    __shared__ uint32_t tmem_s;
    __shared__ int abort_s;
    volatile int* abort = &abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int sl = blockIdx.y, row0 = blockIdx.x * TC_M;
    C += (long)sl * sC;
    const int Mr = OPA == OP_N ? Mc : 2 * Mc;
    const int Kr = OPA == OP_N ? 2 * Kc : Kc;
    const int nkt = (Kr + G::KT - 1) / G::KT;
    // stage ring at a 1024-byte boundary (the 128-byte swizzle repeats every 1024 bytes)
    const uint32_t sbase = (smem_u32(sm_raw) + 1023u) & ~1023u;
    unsigned char* sgen = sm_raw + (sbase - smem_u32(sm_raw));

    if (tid == 0) {
        for (int i = 0; i < ns; ++i) {
            mbar_init_n(smem_u32(&full[i]), 1);
            mbar_init_n(smem_u32(&conv[i]), TC_CONV_WARPS);
            mbar_init_n(smem_u32(&empty[i]), 1);
        }
        mbar_init_n(smem_u32(&accf), 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                     "r"(G::ncols(ns))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_s;

    if (warp == TC_PROD_WARP) {
        if (lane == 0) {
            int issued = 0;
            for (int kt = 0; kt < nkt; ++kt) {
                const int st = kt % ns;
                if (kt >= ns && !mbar_wait(smem_u32(&empty[st]), (uint32_t)((kt / ns - 1) & 1), abort, spin)) break;
                const uint32_t buf = sbase + (uint32_t)(st * G::STAGE);
                const uint32_t fb = smem_u32(&full[st]);
                mbar_expect_tx(fb, G::TX);
                if (OPA == OP_N) tma_load_3d(buf + G::A_RAW, &tmA, kt * G::KT, row0, sl, fb);
                else tma_load_3d(buf + G::A_RAW, &tmA, row0, kt * TC_KT, sl, fb);
                tma_load_3d(buf + G::B_RAW, &tmB, 0, kt * G::KB, sl, fb);
                issued = kt + 1;
            }
            // drain: every TMA write lands before the CTA can end
            for (int kt = issued - ns > 0 ? issued - ns : 0; kt < issued; ++kt)
                mbar_drain(smem_u32(&full[kt % ns]), (uint32_t)((kt / ns) & 1));
        }
    } else if (warp == TC_MMA_WARP) {
        if (lane == 0) {
            const uint32_t id_full = NP == 0 ? idesc_bf16(TC_M, G::NB) : idesc_tf32(TC_M, G::NB);
            const uint32_t id_half = idesc_tf32(TC_M, 2 * NCP);
            // the shared-memory descriptors of stage 0, k-step 0; a stage or k-step
            // only moves the start address (bits 0-13, in 16-byte units), and every
            // operand address is below 228 KB, so the offsets add without a carry
            // out of that field
            const uint64_t da0 = OPA == OP_N ? sdesc(sbase + G::A_HI, 16, TC_SBO_SW, 2)
                                             : sdesc(sbase + G::A_HI, TC_LBO_A, TC_SBO);
            const uint64_t dl0 = OPA == OP_N ? sdesc(sbase + G::A_LO, 16, TC_SBO_SW, 2)
                                             : sdesc(sbase + G::A_LO, TC_LBO_A, TC_SBO);
            const uint64_t db0 = sdesc(sbase + G::B_OP, G::LBO_B, TC_SBO);
            constexpr uint64_t A_KS = OPA == OP_N ? 32 / 16 : 2 * TC_LBO_A / 16;  // per k-step, 16-byte units
            constexpr uint64_t B_KS = 2 * G::LBO_B / 16;
            int issued = 0;
            for (int kt = 0; kt < nkt; ++kt) {
                const int st = kt % ns;
                if (!mbar_wait(smem_u32(&conv[st]), (uint32_t)((kt / ns) & 1), abort, spin)) break;
                tc_fence_after();
                const uint64_t so = (uint64_t)(st * (G::STAGE / 16));
                const uint32_t tlo = tmem + (uint32_t)(G::ACC + 32 * st);
#pragma unroll
                for (int ks = 0; ks < TC_KT / 8; ++ks) {
                    const uint64_t dah = da0 + so + A_KS * ks, dal = dl0 + so + A_KS * ks;
                    const uint64_t db = db0 + so + B_KS * ks;
                    if (NP == 0) {  // 16 bfloat16 reduction entries per step (32 bytes, as 8 tf32)
                        mma_bf16(tmem, dah, db, id_full, (kt > 0 || ks > 0) ? 1u : 0u);
                        continue;
                    }
                    mma_tf32(tmem, dah, db, id_full, (kt > 0 || ks > 0) ? 1u : 0u);  // hi*hi [| hi*lo]
                    if (G::LO_TM)                                                    // += lo*hi
                        mma_tf32_ta(tmem, tlo + (uint32_t)(8 * ks), db, id_half, 1u);
                    else if (NP == 3)
                        mma_tf32(tmem, dal, db, id_half, 1u);
                }
                mma_commit(smem_u32(&empty[st]));
                issued = kt + 1;
            }
            if (issued == nkt) {
                mma_commit(smem_u32(&accf));
            } else if (issued > 0) {  // aborted: let the MMAs in flight finish
                mbar_drain(smem_u32(&empty[(issued - 1) % ns]), (uint32_t)(((issued - 1) / ns) & 1));
            }
        }
    } else {
        // warps 0-7: split each stage, then the epilogue
        for (int kt = 0; kt < nkt; ++kt) {
            const int st = kt % ns;
            if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((kt / ns) & 1), abort, spin)) break;
            split_stage<OPA, CONJ, NCP, NP>(sgen + st * G::STAGE, tmem + (uint32_t)(G::ACC + 32 * st));
            fence_async_smem();  // generic-proxy writes -> tensor-core reads
            if (G::LO_TM) {      // the lo tile's tensor-memory stores complete before the MMA thread reads it
                tmem_st_wait();
                tc_fence_before();
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&conv[st]));
        }
        const bool ok = mbar_wait(smem_u32(&accf), 0u, abort, spin);
        if (__all_sync(0xffffffffu, ok)) {
            tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
            const int r = row0 + 32 * (warp & 3) + lane;  // real row of the MMA
            for (int c0 = 8 * (warp >> 2); c0 < NCP; c0 += 16) {
                // columns c0..c0+7 of the four groups: re (hi*hi + lo*hi), im (...), re (hi*lo), im (hi*lo)
                float d[4][8];
#pragma unroll
                for (int g = 0; g < (NP == 3 ? 4 : 2); ++g) tmem_ld8(ta + (uint32_t)(g * NCP + c0), d[g]);
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    const int c = c0 + cc;
                    const float re = NP == 3 ? d[0][cc] + d[2][cc] : d[0][cc];
                    const float im = NP == 3 ? d[1][cc] + d[3][cc] : d[1][cc];
                    if (OPA == OP_N) {
                        if (r < Mr && c < Nc) C[trans_out ? (long)c * ldc + r : (long)r * ldc + c] = make_float2(re, im);
                    } else {
                        // rows 2j (re of A) and 2j+1 (im of A) sit in neighbouring lanes
                        const float pim = __shfl_xor_sync(0xffffffffu, im, 1);
                        const float v = (lane & 1) ? (pim - re) : (re + pim);
                        if (r < Mr && c < Nc) ((float*)C)[((long)(r >> 1) * ldc + c) * 2 + (r & 1)] = v;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && abort_s && err) atomicExch(err, (int)TP_ERR_TIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::ncols(ns))
                     : "memory");
    }
}

typedef PFN_cuTensorMapEncodeTiled_v12000 EncodeFn;

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)p;
    });
    return fn;
}

// 3-D tensor map over (columns, rows, slices) with the given box; float32
// elements, or bfloat16 when bf16.
bool make_map(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint64_t slices, uint64_t row_bytes,
              uint64_t slice_bytes, uint32_t box_c, uint32_t box_r, bool swz, bool bf16 = false) {
    EncodeFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {cols, rows, slices};
    const cuuint64_t strides[2] = {row_bytes, slice_bytes};
    const cuuint32_t box[3] = {box_c, box_r, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
              const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, swz ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int OPA, bool CONJ, int NCP, int NP>
tp_status launch_tc(int batch, int M, int N, int K, const void* A, long lda, long sA, const void* B, long ldb,
                    long sB, void* C, long ldc, long sC, const int* skip, int* err, int trans_out, const int* ncap,
                    int c0, cudaStream_t st, int ns) {
    typedef TcCfg<OPA, NCP, NP> G;
    if (ns <= 0) ns = G::NS;                       // the built-in rule
    if (ns < 2 || ns > G::NS_FIT) return TP_ERR_UNSUPPORTED;
    const size_t smem = G::smem(ns);
    CUtensorMap ma, mb;
    // A: op N rows i of 2K floats (box 32 x 128, swizzled; bfloat16: 2K entries of 2 bytes, box 64 x 128);
    // op C rows i of 2M floats (box 128 x 32)
    const uint64_t ab = NP == 0 ? 4 : 8;  // bytes per complex entry of A
    const bool oka = OPA == OP_N ? make_map(&ma, A, 2 * (uint64_t)K, M, batch, ab * (uint64_t)lda,
                                            ab * (uint64_t)sA, G::KT, TC_M, true, NP == 0)
                                 : make_map(&ma, A, 2 * (uint64_t)M, K, batch, 8 * (uint64_t)lda,
                                            8 * (uint64_t)sA, TC_M, TC_KT, false);
    const bool okb =
        make_map(&mb, B, 2 * (uint64_t)N, K, batch, 8 * (uint64_t)ldb, 8 * (uint64_t)sB, 2 * NCP, G::KB, false);
    if (!oka || !okb) return TP_ERR_UNSUPPORTED;
    auto kern = k_zgemm_tc<OPA, CONJ, NCP, NP>;
    if (smem_optin((const void*)kern, smem) != TP_OK) return TP_ERR_CUDA;
    const int Mr = OPA == OP_N ? M : 2 * M;
    dim3 grid((unsigned)((Mr + TC_M - 1) / TC_M), (unsigned)batch);
    prof_begin(TP_KC_GEMM, st);
    kern<<<grid, TC_THREADS, smem, st>>>(ma, mb, (float2*)C, ldc, sC, M, N, K, skip, err, trans_out, ncap, c0,
                                          wait_budget(TC_SPIN), ns);
    return launched(TP_KC_GEMM, st);
}

// Deterministic scratch operands for the tuner (values of order one, no denormals).
__global__ void k_tune_fill(float* x, long cnt, float f) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) x[i] = __sinf(f * (float)(i % 8191) + 0.3f);
}
__global__ void k_tune_fill_bf16(__nv_bfloat16* x, long cnt, float f) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) x[i] = __float2bfloat16(__sinf(f * (float)(i % 8191) + 0.3f));
}

// Stage counts picked by the tuner, per product shape.
struct TuneKey {
    int op, passes, ncp, M, K, batch;
    bool operator<(const TuneKey& o) const {
        return std::tie(op, passes, ncp, M, K, batch) < std::tie(o.op, o.passes, o.ncp, o.M, o.K, o.batch);
    }
};
struct TuneVal {
    int ns;
    float ms, ms_default;
    int ns_default;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

int tuned_ns(int op, int passes, int ncp, int M, int K, int batch) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(TuneKey{op, passes, ncp, M, K, batch});
    return it == g_tune.end() ? 0 : it->second.ns;
}

// The kernel's default stage count and the largest one for a shape (0 when the kernel does not take it).
void ns_range(int opA, int passes, int ncp, int* dflt, int* fit) {
    *dflt = *fit = 0;
#define TC_R(OP, P, NC)                     \
    {                                       \
        typedef TcCfg<OP, NC, P> G;         \
        *dflt = G::NS;                      \
        *fit = G::NS_FIT;                   \
    }
#define TC_RS(OP, P)                                   \
    switch (ncp) {                                     \
        case 8: TC_R(OP, P, 8) break;                  \
        case 16: TC_R(OP, P, 16) break;                \
        case 24: TC_R(OP, P, 24) break;                \
        default: TC_R(OP, P, 32) break;                \
    }
    const int op = opA == OP_C ? OP_C : OP_N;
    if (passes == 3) {
        if (op == OP_N) TC_RS(OP_N, 3) else TC_RS(OP_C, 3)
    } else if (passes == 1) {
        if (op == OP_N) TC_RS(OP_N, 1) else TC_RS(OP_C, 1)
    } else if (op == OP_N) {
        TC_RS(OP_N, 0)
    }
#undef TC_RS
#undef TC_R
}

}  // namespace

tp_status zgemm_tc_ns(int batch, int M, int N, int K, const void* A, long lda, long sA, int opA, const void* B,
                      long ldb, long sB, void* C, long ldc, long sC, const int* skip, int* err, int passes,
                      cudaStream_t st, int trans_out, const int* ncap, int c0, int ns);

// Returns TP_ERR_UNSUPPORTED (nothing enqueued) when the shape or alignment
// does not fit this kernel; the caller then uses the SIMT product.  The stage
// count is the tuner's for this shape when it has one, else the built-in rule.
tp_status zgemm_tc(int batch, int M, int N, int K, const void* A, long lda, long sA, int opA, const void* B, long ldb,
                   long sB, void* C, long ldc, long sC, const int* skip, int* err, int passes, cudaStream_t st,
                   int trans_out, const int* ncap, int c0) {
    const int ns = tuned_ns(opA, passes, (N + 7) & ~7, M, K, batch);
    return zgemm_tc_ns(batch, M, N, K, A, lda, sA, opA, B, ldb, sB, C, ldc, sC, skip, err, passes, st, trans_out, ncap,
                       c0, ns);
}

tp_status zgemm_tc_ns(int batch, int M, int N, int K, const void* A, long lda, long sA, int opA, const void* B,
                      long ldb, long sB, void* C, long ldc, long sC, const int* skip, int* err, int passes,
                      cudaStream_t st, int trans_out, const int* ncap, int c0, int ns) {
    if (opA != OP_N && opA != OP_R && opA != OP_C) return TP_ERR_UNSUPPORTED;
    if (passes != 0 && passes != 1 && passes != 3) return TP_ERR_UNSUPPORTED;
    // bfloat16 A (passes 0): op N or R only, rows and slices 16-byte multiples (4 complex entries)
    if (passes == 0 && (opA == OP_C || (lda & 3) || (sA & 3))) return TP_ERR_UNSUPPORTED;
    if (trans_out && opA == OP_C) return TP_ERR_UNSUPPORTED;
    if (batch < 1 || batch > 65535 || M < 1 || N < 1 || N > 32 || K < 1) return TP_ERR_UNSUPPORTED;
    // tensor maps: 16-byte aligned bases and 16-byte multiples for the row and slice strides
    if ((lda & 1) || (sA & 1) || (ldb & 1) || (sB & 1) || ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
        return TP_ERR_UNSUPPORTED;
    if ((opA == OP_C ? 2 * M : M) > 65535 * TC_M) return TP_ERR_UNSUPPORTED;
    const int ncp = (N + 7) & ~7;
#define TC_GO(OP, CJ, NC, P)                                                                                  \
    launch_tc<OP, CJ, NC, P>(batch, M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, skip, err, trans_out, ncap, \
                             c0, st, ns)
#define TC_SWITCH(OP, CJ, P)                          \
    switch (ncp) {                                    \
        case 8: return TC_GO(OP, CJ, 8, P);           \
        case 16: return TC_GO(OP, CJ, 16, P);         \
        case 24: return TC_GO(OP, CJ, 24, P);         \
        default: return TC_GO(OP, CJ, 32, P);         \
    }
    if (passes == 3) {
        if (opA == OP_N) TC_SWITCH(OP_N, false, 3)
        if (opA == OP_R) TC_SWITCH(OP_N, true, 3)
        TC_SWITCH(OP_C, false, 3)
    }
    if (passes == 0) {
        if (opA == OP_N) TC_SWITCH(OP_N, false, 0)
        TC_SWITCH(OP_N, true, 0)
    }
    if (opA == OP_N) TC_SWITCH(OP_N, false, 1)
    if (opA == OP_R) TC_SWITCH(OP_N, true, 1)
    TC_SWITCH(OP_C, false, 1)
#undef TC_SWITCH
#undef TC_GO
}

// Times every stage count from 2 to the largest that fits for one product
// shape on scratch operands (filled here; A is M x K, B K x N, C M x N per
// slice, row-major, bfloat16 A for passes 0) and records the fastest.
// Synchronises the stream.  TP_ERR_UNSUPPORTED when the kernel does not take
// the shape, TP_ERR_WORKSPACE when the scratch is too small.
tp_status zgemm_tc_tune(int batch, int M, int N, int K, int opA, int passes, int trans_out, void* scratch,
                        size_t scratch_bytes, cudaStream_t st, int* ns_out, float* ms_out, float* ms_dflt) {
    const int ncp = (N + 7) & ~7;
    int dflt = 0, fit = 0;
    ns_range(opA, passes, ncp, &dflt, &fit);
    if (dflt == 0) return TP_ERR_UNSUPPORTED;
    const long rows = opA == OP_C ? K : M, cols = opA == OP_C ? M : K;  // A stored rows x cols complex
    const size_t ab = passes == 0 ? 4 : 8;
    const size_t a_bytes = (((size_t)batch * rows * cols * ab) + 255) & ~(size_t)255;
    const size_t b_bytes = (((size_t)batch * K * N * 8) + 255) & ~(size_t)255;
    const size_t c_bytes = (size_t)batch * M * N * 8;
    if (!scratch || ((uintptr_t)scratch & 255) || scratch_bytes < a_bytes + b_bytes + c_bytes) return TP_ERR_WORKSPACE;
    unsigned char* base = (unsigned char*)scratch;
    void *A = base, *B = base + a_bytes, *C = base + a_bytes + b_bytes;
    const long na = (long)batch * rows * cols * 2, nb = (long)batch * K * N * 2;
    if (passes == 0) k_tune_fill_bf16<<<(unsigned)((na + 255) / 256), 256, 0, st>>>((__nv_bfloat16*)A, na, 0.37f);
    else k_tune_fill<<<(unsigned)((na + 255) / 256), 256, 0, st>>>((float*)A, na, 0.37f);
    k_tune_fill<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>((float*)B, nb, 0.71f);
    if (cudaGetLastError() != cudaSuccess) return TP_ERR_CUDA;
    const long ldc = trans_out ? M : N;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TP_ERR_CUDA;
    int best = 0;
    float best_ms = 0.f, d_ms = 0.f;
    tp_status err = TP_OK;
    for (int ns = 2; ns <= fit && err == TP_OK; ++ns) {
        auto run = [&]() {
            return zgemm_tc_ns(batch, M, N, K, A, cols, rows * cols, opA, B, N, (long)K * N, C, ldc, (long)M * N,
                               nullptr, nullptr, passes, st, trans_out, nullptr, 0, ns);
        };
        for (int w = 0; w < 2 && err == TP_OK; ++w) err = run();
        if (err != TP_OK) break;
        float ms = 1e30f;
        for (int rep = 0; rep < 5 && err == TP_OK; ++rep) {  // the fastest of five launches
            cudaEventRecord(e0, st);
            err = run();
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) err = TP_ERR_CUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = t < ms ? t : ms;
        }
        if (ns == dflt) d_ms = ms;
        if (best == 0 || ms < best_ms) {
            best = ns;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != TP_OK) return err;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[TuneKey{opA, passes, ncp, M, K, batch}] = TuneVal{best, best_ms, d_ms, dflt};
    }
    if (ns_out) *ns_out = best;
    if (ms_out) *ms_out = best_ms;
    if (ms_dflt) *ms_dflt = d_ms;
    return TP_OK;
}

// The tuner's table: up to max entries (op, passes, columns, M, K, batch, stages, ms, default stages,
// default ms) into out as ints and floats; returns the number of entries.
int zgemm_tc_tuned(int* ints, float* flts, int max) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    int i = 0;
    for (const auto& kv : g_tune) {
        if (i >= max) break;
        int* o = ints + 8 * i;
        o[0] = kv.first.op;
        o[1] = kv.first.passes;
        o[2] = kv.first.ncp;
        o[3] = kv.first.M;
        o[4] = kv.first.K;
        o[5] = kv.first.batch;
        o[6] = kv.second.ns;
        o[7] = kv.second.ns_default;
        flts[2 * i] = kv.second.ms;
        flts[2 * i + 1] = kv.second.ms_default;
        ++i;
    }
    return i;
}

// Sets the stage count of one product shape (op as zgemm_tc takes it, columns
// before rounding); TP_ERR_UNSUPPORTED outside 2 .. the largest that fits.
tp_status zgemm_tc_set(int op, int passes, int N, int M, int K, int batch, int ns) {
    const int ncp = (N + 7) & ~7;
    int dflt = 0, fit = 0;
    ns_range(op, passes, ncp, &dflt, &fit);
    if (dflt == 0 || ns < 2 || ns > fit) return TP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[TuneKey{op, passes, ncp, M, K, batch}] = TuneVal{ns, 0.f, 0.f, dflt};
    return TP_OK;
}

void zgemm_tc_untune() {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
}

}  // namespace tp
