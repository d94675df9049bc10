// Device-side codecs and compensated accumulation of the reduced-precision float
// payloads, shared by the quantised all-reduce and the batched collective engine.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace shmemg {

// ---------------------------------------------------------------- codecs
// E4M3 decode from the format: 1 sign, 4 exponent bits (bias 7), 3 mantissa bits;
// exponent field 0 holds subnormals m/8 * 2^-6 (exact in binary32).
__device__ __forceinline__ float e4m3_decode(uint32_t q) {
    const uint32_t s = (q >> 7) & 1u, e = (q >> 3) & 15u, m = q & 7u;
    float v;
    if (e == 0) {
        v = (float)m * 0.001953125f;  // m * 2^-9, exact
    } else {
        v = __uint_as_float(((e + 120u) << 23) | (m << 20));  // (1 + m/8) * 2^(e-7)
    }
    return s ? -v : v;
}
__device__ __forceinline__ float bf16_decode(uint32_t q) { return __uint_as_float(q << 16); }

// two floats -> two E4M3 codes (round to nearest even, saturate to +-448); `lo` is the
// element at the lower address
__device__ __forceinline__ uint16_t e4m3x2_encode(float lo, float hi) {
    uint16_t r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ uint16_t bf16_encode(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// ---------------------------------------------------------------- compensated sum
// Neumaier: t = sum + x; c += (sum - t) + x if |sum| >= |x| else (x - t) + sum; sum = t.
struct Neu {
    float sum, c;
    __device__ __forceinline__ void add(float x) {
        const float t = __fadd_rn(sum, x);
        if (fabsf(sum) >= fabsf(x)) c = __fadd_rn(c, __fadd_rn(__fsub_rn(sum, t), x));
        else c = __fadd_rn(c, __fadd_rn(__fsub_rn(x, t), sum));
        sum = t;
    }
    __device__ __forceinline__ float result() const { return __fadd_rn(sum, c); }
};

// Pairs of binary32 values in one 64-bit register (the lower-addressed element in the low
// half) and Blackwell's packed f32x2 arithmetic: two independent IEEE operations, round
// to nearest even, subnormals kept.
__device__ __forceinline__ uint64_t f2(float lo, float hi) {
    return (uint64_t)__float_as_uint(lo) | ((uint64_t)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float f2_lo(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float f2_hi(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// Two compensated sums side by side, Neumaier's step on each: t = sum + x, then c gains
// (a - t) + b with a the larger of sum and x in magnitude (sum when equal) and b the
// other -- the same operations as Neu, the magnitude ordering per lane, the three adds
// packed.
struct Neu2 {
    uint64_t sum, c;
    __device__ __forceinline__ void add(uint64_t x) {
        const uint64_t t = f2_add(sum, x);
        const float s0 = f2_lo(sum), s1 = f2_hi(sum), x0 = f2_lo(x), x1 = f2_hi(x);
        const bool g0 = fabsf(s0) >= fabsf(x0), g1 = fabsf(s1) >= fabsf(x1);
        const uint64_t a = f2(g0 ? s0 : x0, g1 ? s1 : x1), b = f2(g0 ? x0 : s0, g1 ? x1 : s1);
        c = f2_add(c, f2_add(f2_sub(a, t), b));
        sum = t;
    }
    __device__ __forceinline__ uint64_t result() const { return f2_add(sum, c); }
};

// Elements per thread of the wide path: one 16-byte code load per member.
template <int FMT> struct QWide { static constexpr int E = FMT == SHMEMG_FMT_E4M3 ? 16 : 8; };

// The E dequantised values of one 16-byte code load, as E/2 pairs: decoded exactly to
// binary32, then one RNE multiply by the block scale each (packed).
template <int FMT>
__device__ __forceinline__ void qdecode16(uint4 w, float s, uint64_t *d) {
    const uint32_t v[4] = {w.x, w.y, w.z, w.w};
    const uint64_t ss = f2(s, s);
    if (FMT == SHMEMG_FMT_E4M3) {
        // hardware conversion of code pairs to f16 (exact: every E4M3 value is an f16
        // value), then to binary32
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
            const uint16_t pair = (uint16_t)((v[j >> 2] >> (8 * (j & 3))) & 0xFFFFu);
            uint32_t h2;
            asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(pair));
            d[j >> 1] = f2_mul(f2(__half2float(__ushort_as_half((unsigned short)(h2 & 0xFFFFu))),
                                  __half2float(__ushort_as_half((unsigned short)(h2 >> 16)))),
                               ss);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) d[j] = f2_mul(f2(bf16_decode(v[j] & 0xFFFFu), __uint_as_float(v[j] & 0xFFFF0000u)), ss);
    }
}

// Wide form of qsum4: elements [e0, e0+E) with E = QWide<FMT>::E, e0 a multiple of E,
// q_off and d_off 16-byte aligned, e0 + E <= n.  M members' codes and scales are
// loaded ahead of their accumulation, which stays in team-rank order.
template <int FMT, int M = 8>
__device__ __forceinline__ void qsum_wide_acc(const uint8_t *heap, uint64_t H, int pe0, int pstride, int P,
                                              uint64_t q_off, uint64_t s_off, uint64_t e0, float4 *o);

template <int FMT, int M = 8>
__device__ __forceinline__ void qsum_wide(uint8_t *heap, uint64_t H, int pe0, int pstride, int P, uint64_t d_off,
                                          uint64_t q_off, uint64_t s_off, uint64_t e0) {
    constexpr int E = QWide<FMT>::E;
    float4 o[E / 4];
    qsum_wide_acc<FMT, M>(heap, H, pe0, pstride, P, q_off, s_off, e0, o);
    for (int m = 0; m < P; m++) {
        float4 *dst = (float4 *)(heap + (uint64_t)(pe0 + m * pstride) * H + d_off + 4 * e0);
#pragma unroll
        for (int k = 0; k < E / 4; k++) dst[k] = o[k];
    }
}

// The accumulation of qsum_wide: the E compensated sums of elements [e0, e0+E) into o;
// M members' codes and scales are loaded ahead.
template <int FMT, int M>
__device__ __forceinline__ void qsum_wide_acc(const uint8_t *heap, uint64_t H, int pe0, int pstride, int P,
                                              uint64_t q_off, uint64_t s_off, uint64_t e0, float4 *o) {
    constexpr int E = QWide<FMT>::E;
    constexpr uint64_t QS = FMT == SHMEMG_FMT_E4M3 ? 1 : 2;
    Neu2 acc[E / 2];
#pragma unroll
    for (int j = 0; j < E / 2; j++) acc[j] = {0ull, 0ull};
    uint64_t d[E / 2];
    int r = 0;
    for (; r + M <= P; r += M) {
        uint4 w[M];
        float sc[M];
#pragma unroll
        for (int u = 0; u < M; u++) {
            const uint8_t *b = heap + (uint64_t)(pe0 + (r + u) * pstride) * H;
            w[u] = __ldcg((const uint4 *)(b + q_off + e0 * QS));
            sc[u] = __ldcg((const float *)(b + s_off) + e0 / 128);
        }
#pragma unroll
        for (int u = 0; u < M; u++) {
            qdecode16<FMT>(w[u], sc[u], d);
#pragma unroll
            for (int j = 0; j < E / 2; j++) acc[j].add(d[j]);
        }
    }
    for (; r < P; r++) {
        const uint8_t *b0 = heap + (uint64_t)(pe0 + r * pstride) * H;
        qdecode16<FMT>(__ldcg((const uint4 *)(b0 + q_off + e0 * QS)), __ldcg((const float *)(b0 + s_off) + e0 / 128), d);
#pragma unroll
        for (int j = 0; j < E / 2; j++) acc[j].add(d[j]);
    }
#pragma unroll
    for (int k = 0; k < E / 4; k++) {
        const uint64_t a = acc[2 * k].result(), b = acc[2 * k + 1].result();
        o[k] = make_float4(f2_lo(a), f2_hi(a), f2_lo(b), f2_hi(b));
    }
}

// One CTA's chunk of blockDim.x * E elements starting at c0 (full, aligned): every thread
// accumulates its E elements into shared memory, then thread 0 bulk-stores the chunk to
// every member (one TMA store per member instead of P x E/4 vector stores per thread).
// `out` holds blockDim.x * E floats (128-byte aligned); callers alternate two such
// buffers.  The bulk stores of the previous chunks drain while this chunk is loaded and
// accumulated; before `out` is overwritten thread 0 waits only until every bulk group but
// the most recent one (the previous chunk's, from the other buffer) has read its source
// (bulk wait_group.read 1).  Returns with the stores issued as one bulk group.
template <int FMT, int M = 8>
__device__ __forceinline__ void qsum_chunk_tma(uint8_t *heap, uint64_t H, int pe0, int pstride, int P, uint64_t d_off,
                                               uint64_t q_off, uint64_t s_off, uint64_t c0, float *out) {
    constexpr int E = QWide<FMT>::E;
    float4 o[E / 4];
    qsum_wide_acc<FMT, M>(heap, H, pe0, pstride, P, q_off, s_off, c0 + (uint64_t)threadIdx.x * E, o);
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");  // `out` free again
    __syncthreads();
#pragma unroll
    for (int k = 0; k < E / 4; k++) reinterpret_cast<float4 *>(out)[threadIdx.x * (E / 4) + k] = o[k];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic smem writes -> bulk copy engine
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bytes = blockDim.x * E * 4;
        for (int m = 0; m < P; m++)
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(
                             heap + (uint64_t)(pe0 + m * pstride) * H + d_off + 4 * c0),
                         "r"((uint32_t)__cvta_generic_to_shared(out)), "r"(bytes)
                         : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
}

// Dequantised sum of elements [e0, e0+4) over the team members, written to every
// member's dst.  Vector path: 4 codes and 4 floats per access (aligned offsets).
template <int FMT>
__device__ __forceinline__ void qsum4(uint8_t *heap, uint64_t H, int pe0, int pstride, int P, uint64_t d_off,
                                      uint64_t q_off, uint64_t s_off, uint64_t e0, uint64_t n, bool vec) {
    Neu acc[4];
#pragma unroll
    for (int j = 0; j < 4; j++) acc[j] = {0.0f, 0.0f};
    for (int r = 0; r < P; r++) {
        const uint8_t *base = heap + (uint64_t)(pe0 + r * pstride) * H;
        float d[4];
        if (vec) {
            const float s = __ldcg((const float *)(base + s_off) + e0 / 128);
            if (FMT == SHMEMG_FMT_E4M3) {
                const uint32_t w = __ldcg((const unsigned int *)(base + q_off + e0));
#pragma unroll
                for (int j = 0; j < 4; j++) d[j] = __fmul_rn(e4m3_decode((w >> (8 * j)) & 0xFFu), s);
            } else {
                const uint2 w = __ldcg((const uint2 *)(base + q_off + 2 * e0));
                d[0] = __fmul_rn(bf16_decode(w.x & 0xFFFFu), s);
                d[1] = __fmul_rn(bf16_decode(w.x >> 16), s);
                d[2] = __fmul_rn(bf16_decode(w.y & 0xFFFFu), s);
                d[3] = __fmul_rn(bf16_decode(w.y >> 16), s);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint64_t e = e0 + j;
                if (e >= n) { d[j] = 0.0f; continue; }
                const float s = ((const float *)(base + s_off))[e / 128];
                const float v = FMT == SHMEMG_FMT_E4M3 ? e4m3_decode(base[q_off + e])
                                                       : bf16_decode(((const uint16_t *)(base + q_off))[e]);
                d[j] = __fmul_rn(v, s);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) acc[j].add(d[j]);
    }
    if (vec) {
        const float4 o = make_float4(acc[0].result(), acc[1].result(), acc[2].result(), acc[3].result());
        for (int r = 0; r < P; r++) *(float4 *)(heap + (uint64_t)(pe0 + r * pstride) * H + d_off + 4 * e0) = o;
    } else {
        for (int r = 0; r < P; r++) {
            float *dst = (float *)(heap + (uint64_t)(pe0 + r * pstride) * H + d_off);
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (e0 + j < n) dst[e0 + j] = acc[j].result();
        }
    }
}

}  // namespace shmemg
