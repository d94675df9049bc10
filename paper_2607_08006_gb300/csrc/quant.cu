// Reduced-precision float payloads for the sum all-reduce (a precision extension; the
// paper's reductions are inherited from OpenSHMEM 1.6, Sec. 6.3): per-128-element
// block scales, bf16 or OCP FP8 E4M3 codes, dequantised and accumulated in binary32
// with Neumaier compensated summation in team-rank order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "quant_dev.cuh"

namespace shmemg {

constexpr int Q_THREADS = 256;

// ---------------------------------------------------------------- quantize
// One warp per 128-element block: lane l owns elements 4l..4l+3 of the block.
struct QArgs {
    uint8_t *heap;
    uint64_t H;
    int start, stride, size;
    uint64_t q_off, s_off, x_off;
    uint64_t n;
    int fmt;
};

__global__ void __launch_bounds__(Q_THREADS) k_quantize(QArgs a) {
    const uint64_t nblk = (a.n + 127) / 128;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t wid = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const float R = a.fmt == SHMEMG_FMT_E4M3 ? 448.0f : 1.0f;
    const uint64_t total = nblk * (uint64_t)a.size;
    for (uint64_t it = wid; it < total; it += warps) {
        const int r = (int)(it / nblk);
        const uint64_t b = it - (uint64_t)r * nblk;
        uint8_t *base = a.heap + (uint64_t)(a.start + r * a.stride) * a.H;
        const float *x = (const float *)(base + a.x_off);
        const uint64_t e0 = b * 128 + (uint64_t)lane * 4;
        float v[4];
        const bool full = (b + 1) * 128 <= a.n && ((a.x_off & 15) == 0);
        if (full) {
            float4 t = __ldcs((const float4 *)(x + e0));
            v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) v[j] = e0 + j < a.n ? x[e0 + j] : 0.0f;
        }
        float am = fmaxf(fmaxf(fabsf(v[0]), fabsf(v[1])), fmaxf(fabsf(v[2]), fabsf(v[3])));
        uint32_t amb = __reduce_max_sync(0xffffffffu, __float_as_uint(am));  // |x| bits order like values
        const float amax = __uint_as_float(amb);
        const float s = amax == 0.0f ? 1.0f : __fdiv_rn(amax, R);
        float y[4];
#pragma unroll
        for (int j = 0; j < 4; j++) y[j] = __fdiv_rn(v[j], s);
        if (lane == 0) ((float *)(base + a.s_off))[b] = s;
        if (a.fmt == SHMEMG_FMT_E4M3) {
            uint8_t *q = base + a.q_off;
            const uint32_t w = (uint32_t)e4m3x2_encode(y[0], y[1]) | ((uint32_t)e4m3x2_encode(y[2], y[3]) << 16);
            if (full && ((a.q_off & 3) == 0)) {
                *(uint32_t *)(q + e0) = w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (e0 + j < a.n) q[e0 + j] = (uint8_t)(w >> (8 * j));
            }
        } else {
            uint16_t *q = (uint16_t *)(base + a.q_off);
            if (full && ((a.q_off & 7) == 0)) {
                uint2 w;
                w.x = (uint32_t)bf16_encode(y[0]) | ((uint32_t)bf16_encode(y[1]) << 16);
                w.y = (uint32_t)bf16_encode(y[2]) | ((uint32_t)bf16_encode(y[3]) << 16);
                *(uint2 *)(q + e0) = w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (e0 + j < a.n) q[e0 + j] = bf16_encode(y[j]);
            }
        }
    }
}

struct QSumArgs {
    uint8_t *heap;
    uint64_t H;
    int start, stride, size, gstride;
    uint64_t d_off, q_off, s_off;
    uint64_t n;
    bool vec;   // 4-element vector path allowed
    bool wide;  // 16-byte code path allowed
};

// Full, aligned chunks of blockDim x E elements: each thread accumulates E elements
// (one 16-byte code load per member) into shared memory and thread 0 bulk-stores the
// chunk to every member (two chunk buffers, so one chunk's stores drain while the next
// is accumulated).  The ragged tail runs in 4-element steps.
template <int FMT>
__global__ void __launch_bounds__(Q_THREADS) k_qsum(QSumArgs a) {
    constexpr int E = QWide<FMT>::E;
    __shared__ __align__(128) float s_out[2][Q_THREADS * E];   // alternate chunk buffers
    const int pe0 = a.start + blockIdx.y * a.gstride;
    const uint64_t CH = (uint64_t)blockDim.x * E;
    const uint64_t nfull = a.wide ? a.n / CH : 0;
    int buf = 0;
    for (uint64_t ch = blockIdx.x; ch < nfull; ch += gridDim.x) {
        qsum_chunk_tma<FMT>(a.heap, a.H, pe0, a.stride, a.size, a.d_off, a.q_off, a.s_off, ch * CH, s_out[buf]);
        buf ^= 1;
    }
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    const uint64_t t0 = nfull * CH;
    for (uint64_t f = t0 + 4 * ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x); f < a.n;
         f += 4 * (uint64_t)gridDim.x * blockDim.x)
        qsum4<FMT>(a.heap, a.H, pe0, a.stride, a.size, a.d_off, a.q_off, a.s_off, f, a.n, a.vec && f + 4 <= a.n);
}

}  // namespace shmemg

using namespace shmemg;

extern "C" {

int shmemg_quantize(shmemg_team_t team, void *q, float *scales, const float *src, int fmt, uint64_t n, void *stream) {
    if (int rc = check_init()) return rc;
    HostTeam t;
    if (team_get(team, &t)) return SHMEMG_ERR_INVALID_ARG;
    if (fmt != SHMEMG_FMT_BF16 && fmt != SHMEMG_FMT_E4M3) return SHMEMG_ERR_INVALID_ARG;
    const uint64_t qs = fmt == SHMEMG_FMT_E4M3 ? 1 : 2, nb = (n + 127) / 128;
    uint64_t qo, so, xo;
    if (sym_offset(q, n * qs, &qo) || sym_offset(scales, nb * 4, &so) || sym_offset(src, n * 4, &xo))
        return SHMEMG_ERR_NOT_SYMMETRIC;
    if ((so & 3) || (xo & 3) || (qo % qs)) return SHMEMG_ERR_INVALID_ARG;
    if (n == 0) return SHMEMG_SUCCESS;
    State &S = st();
    QArgs a;
    a.heap = S.heap;
    a.H = S.H;
    a.q_off = qo;
    a.s_off = so;
    a.x_off = xo;
    a.n = n;
    a.fmt = fmt;
    a.stride = t.stride;
    a.size = t.size;
    int cap = ctas_for((const void *)k_quantize, Q_THREADS, 0);
    for (int g = 0; g < t.ngroups; g++) {
        a.start = t.start + g * t.gstride;
        uint64_t warps = nb * (uint64_t)t.size;
        uint64_t blocks = (warps + (Q_THREADS / 32) - 1) / (Q_THREADS / 32);
        k_quantize<<<(unsigned)(blocks < (uint64_t)cap ? blocks : cap), Q_THREADS, 0, to_stream(stream)>>>(a);
    }
    return cuda_rc(cudaGetLastError());
}

int shmemg_qsum_reduce(shmemg_team_t team, float *dst, const void *q, const float *scales, int fmt, uint64_t n,
                       void *stream) {
    if (int rc = check_init()) return rc;
    HostTeam t;
    if (team_get(team, &t)) return SHMEMG_ERR_INVALID_ARG;
    if (fmt != SHMEMG_FMT_BF16 && fmt != SHMEMG_FMT_E4M3) return SHMEMG_ERR_INVALID_ARG;
    const uint64_t qs = fmt == SHMEMG_FMT_E4M3 ? 1 : 2, nb = (n + 127) / 128;
    uint64_t qo, so, d;
    if (sym_offset(q, n * qs, &qo) || sym_offset(scales, nb * 4, &so) || sym_offset(dst, n * 4, &d))
        return SHMEMG_ERR_NOT_SYMMETRIC;
    if ((so & 3) || (d & 3) || (qo % qs)) return SHMEMG_ERR_INVALID_ARG;
    // dst must not overlap the payload or the scales (they are read by other threads)
    if ((d < qo + n * qs && qo < d + n * 4) || (d < so + nb * 4 && so < d + n * 4)) return SHMEMG_ERR_INVALID_ARG;
    if (n == 0) return SHMEMG_SUCCESS;
    State &S = st();
    QSumArgs a;
    a.heap = S.heap;
    a.H = S.H;
    a.start = t.start;
    a.stride = t.stride;
    a.size = t.size;
    a.gstride = t.gstride;
    a.d_off = d;
    a.q_off = qo;
    a.s_off = so;
    a.n = n;
    a.vec = (d & 15) == 0 && (qo & (fmt == SHMEMG_FMT_E4M3 ? 3 : 7)) == 0;
    a.wide = (d & 15) == 0 && (qo & 15) == 0;
    const void *kfn = fmt == SHMEMG_FMT_E4M3 ? (const void *)k_qsum<SHMEMG_FMT_E4M3> : (const void *)k_qsum<SHMEMG_FMT_BF16>;
    const uint64_t E = fmt == SHMEMG_FMT_E4M3 ? 16 : 8;
    const uint64_t need = (n + Q_THREADS * E - 1) / (Q_THREADS * E);
    dim3 grid((unsigned)balanced_grid(need, (uint64_t)ctas_for(kfn, Q_THREADS, 0), t.ngroups), (unsigned)t.ngroups);
    if (fmt == SHMEMG_FMT_E4M3) k_qsum<SHMEMG_FMT_E4M3><<<grid, Q_THREADS, 0, to_stream(stream)>>>(a);
    else k_qsum<SHMEMG_FMT_BF16><<<grid, Q_THREADS, 0, to_stream(stream)>>>(a);
    return cuda_rc(cudaGetLastError());
}

}  // extern "C"
